// C-ABI of librafem (declared in include/rafem.h): context lifetime, per-step assembly + solve, CUDA-graph
// time loop. The step follows the main loop of Sec. II-A: every corrector pass recomputes the element
// equations with the newest values, assembles the global systems and solves them; here the whole step stays on
// the device, so the per-pass host<->device copies of Sec. III-A (matrix to the host solver, solution back for
// the host-side predictor and convergence check) do not exist.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "setup.h"

using namespace rafem;

namespace {

struct StatsDev {
    rafem_step_stats cur;   // statistics of the step in progress / last step
    int32_t worst;          // worst status over all steps since the last reset
    int32_t hist;           // steps completed since the last state reset (predictor history)
};

struct CorrDev {
    int32_t pass;           // corrector passes done in the current step
    int32_t converged;      // 1 once max |T^{k+1} - T^k| < corrector_tol
    double change;          // max |T^{k+1} - T^k| of the last pass
    double newton_rr;       // monolithic step: ||R||^2 of the last Newton linear solve (0 before the first)
};

}  // namespace

struct rafem_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    rafem_params prm{};
    int N = 0, E = 0;
    int64_t nnz = 0;
    int n_colors = 0;
    std::vector<int> color_off;      // [n_colors + 1] over the sorted element order
    std::vector<void*> allocs;

    // pattern: CSR (rp, ci) or SELL-32 (rp = slice pointers, ci = slice columns) on the device; the CSR
    // pattern and the CSR -> storage map stay on the host for inspection
    int32_t *rp = nullptr, *ci = nullptr, *diag = nullptr;
    int16_t* ci16 = nullptr;  // SELL column deltas (when they fit 16 bits)
    int32_t *pat_off = nullptr, *pat_pool = nullptr;  // one column pattern per slice (kernel code 3)
    bool sell = true;
    int64_t nnz_store = 0;
    std::vector<int32_t> h_rp, h_col, h_map;
    // element data
    ElemData el;
    int32_t* e_nodes = nullptr;
    int32_t* e_slots = nullptr;
    double *e_G = nullptr, *e_vol = nullptr, *e_sig0 = nullptr, *e_k = nullptr;
    double* xyz = nullptr;
    // boundary data
    uint8_t *bcV = nullptr, *bcT = nullptr;
    double *gV = nullptr, *gT = nullptr;
    // systems
    double *valsV = nullptr, *valsT = nullptr;
    float *valsV32 = nullptr, *valsT32 = nullptr;
    double *bV = nullptr, *bT = nullptr, *bTc = nullptr;
    // fields
    double *V = nullptr, *T = nullptr, *T_old = nullptr, *T_prev = nullptr;
    double *V_hist = nullptr, *T_hist = nullptr;   // predictor history (x^{n-1})
    double *V_hist2 = nullptr, *T_hist2 = nullptr; // predictor history (x^{n-2}), quadratic and cubic predictors
    double *V_hist3 = nullptr, *T_hist3 = nullptr; // predictor history (x^{n-3}), cubic predictor and projection
    double* proj_partial = nullptr;                // [kProjQ][n_tiles * proj_sub] projection sums
    int proj_sub = 1;
    double* proj_coef = nullptr;                   // [kProjMax n_inst]
    int proj_k = kProjDefault;                     // basis size limit
    int32_t *proj_kin = nullptr, *proj_kout = nullptr;
    double* proj_D = nullptr;                      // [N][proj_stride(proj_k)] projection basis (its history)
    double* proj_Y = nullptr;                      // [N][proj_stride(proj_k)] A times the basis
    double* proj_r0 = nullptr;                     // [N] residual of the projected guess
    bool r0_fresh = false;                         // enqueue time: proj_r0 belongs to the next potential solve
    // solver workspace
    double *wr = nullptr, *wu = nullptr, *ww = nullptr, *wp = nullptr, *ws = nullptr, *wdinv = nullptr;
    float *fr = nullptr, *fu = nullptr, *fw = nullptr, *fp = nullptr, *fs = nullptr, *fd = nullptr, *fdinv = nullptr;
    double *pz = nullptr, *pq = nullptr, *pm0 = nullptr, *pm1 = nullptr;  // pipelined CG workspace
    int32_t *tile_r0 = nullptr, *tile_r1 = nullptr, *tile_inst = nullptr, *inst_t0 = nullptr, *inst_t1 = nullptr;
    int n_tiles = 0, grid = 0, block = 0, lanes = 8;
    InstState* instV = nullptr;        // [n_inst]
    InstState* instT = nullptr;        // [n_inst]
    int n_inst = 1;                    // independent problem instances (a batch) in this context
    int maxb = 0;                      // co-resident blocks of the solver kernel
    int rows_per_tile = 0;
    std::vector<void*> tile_allocs;    // tile arrays and partial sums (rebuilt by rafem_set_schedule)
    std::vector<int32_t> inst_node_off;  // [n_inst + 1] first node of each instance (multiples of 32)
    rafem_step_stats* istats = nullptr;  // [n_inst] per-instance statistics of the current step
    double* partial = nullptr;
    GridBarrier* bar = nullptr;
    StatsDev* stats = nullptr;
    double* scratch = nullptr;       // small device scratch (max |dT|)
    int64_t step = 0;
    // row-owner assembly
    bool gather = false;
    GatherData gd;
    bool dw = false;  // double-word element and node passes (RAFEM_ARITH_DW resolved at create)
    GatherDw gdw;
    CoupledGather mg;  // coupled Jacobian by rows (monolithic contexts with the gather assembly)
    uint8_t* gather_cg = nullptr;
    long long gather_nc = 0;
    // graph
    cudaGraphExec_t graph = nullptr;
    int32_t graph_kernels = 0;  // kernel nodes of the captured step graph
    bool graph_failed = false;
    // corrector passes (n_corrector > 1): one graph per step whose conditional WHILE node repeats the pass on the
    // device until the temperature change falls below corrector_tol or n_corrector passes are done
    cudaGraphExec_t corr_graph = nullptr;
    // host-state step (rafem_step_host): copies on a second stream, overlapped with the step, captured as a graph
    // for one set of host buffers
    cudaStream_t io_stream = nullptr;
    cudaEvent_t io_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t io_graph = nullptr;
    bool io_graph_failed = false;
    const void* io_key[4] = {nullptr, nullptr, nullptr, nullptr};
    bool corr_graph_failed = false;
    CorrDev* corr = nullptr;
    double* V_old = nullptr;          // potential at the start of the step (restored when a step is rejected)
    StatsDev* stats_save = nullptr;   // statistics at the start of the step (idem)
    rafem_step_stats* istats_save = nullptr;
    // tracing
    bool tracing = false;
    rafem_trace trace{};
    cudaEvent_t ev[8] = {};
    // ILU(0) preconditioner (precond == RAFEM_PRECOND_ILU0)
    bool ilu = false;
    IluLayout il;
    std::vector<int32_t> ilu_pmap_csr;   // [nnz_p] CSR position of each factor entry (host), < 0 none
    std::vector<int32_t> ilu_perm;       // [Np] original row of each padded row (host), -1 dummy
    double *ilu_AV = nullptr, *ilu_FV = nullptr, *ilu_AT = nullptr, *ilu_FT = nullptr;
    double *ilu_DV = nullptr, *ilu_DT = nullptr;  // 1 / diag(U)
    IluRingDev ir[2];                    // ring ILU solver: layouts and workspace shared, values per system (V, T)
    int ir_grid = 0;
    // BiCGSTAB (solver == RAFEM_SOLVER_BICGSTAB)
    double *bg_r = nullptr, *bg_rh = nullptr, *bg_p = nullptr, *bg_ph = nullptr, *bg_v = nullptr, *bg_s = nullptr,
           *bg_sh = nullptr, *bg_t = nullptr, *bg_dinv = nullptr, *bg_partial = nullptr;
    int bg_grid = 0;
    // GMRES(m) (solver == RAFEM_SOLVER_GMRES)
    int gm_m = 0, gm_grid = 0;
    // monolithic coupled step (coupling == RAFEM_COUPLING_MONOLITHIC): 2 x 2 block Jacobian on the node pattern,
    // interleaved residual and Newton correction, block-BiCGSTAB workspace (2N vectors)
    bool mono = false;
    double *m_vals4 = nullptr, *m_R = nullptr, *m_D = nullptr;
    double *mb_r = nullptr, *mb_rh = nullptr, *mb_p = nullptr, *mb_ph = nullptr, *mb_v = nullptr, *mb_s = nullptr,
           *mb_sh = nullptr, *mb_t = nullptr, *mb_dinv = nullptr, *mb_partial = nullptr;
    int mb_grid = 0;
    // flexible GMRES of the monolithic step (coupled_solver = RAFEM_COUPLED_FGMRES): basis V (kFgMax + 1 vectors
    // of 2N) and preconditioned vectors Z (kFgMax), the Arnoldi vector, the split preconditioner's vectors
    double *fg_V = nullptr, *fg_Z = nullptr, *fg_w = nullptr, *fg_partial = nullptr;
    double *fg_rV = nullptr, *fg_rT = nullptr, *fg_zV = nullptr, *fg_zT = nullptr;
    FgState* fg_st = nullptr;
    int32_t* fg_one = nullptr;  // [1] = 1: the inner solves' starting residual is given (x0 = 0, r0 = b)
    size_t fg_ld = 0;
    int fg_G = 0;
    double *gm_V = nullptr, *gm_w0 = nullptr, *gm_w1 = nullptr, *gm_dinv = nullptr, *gm_partial = nullptr;
    double *gm_z = nullptr, *gm_H = nullptr;  // M^-1 of the next SpMV's input; per-block Hessenberg copies
    int gm_ld = 0;                            // row stride of the basis
    // differentiation: element order map, tape of checkpoints, adjoint workspace
    int32_t* e_order = nullptr;      // [E] stored element -> mesh element
    int32_t* e_clist = nullptr;      // [E] stored elements in colour order (row-owner assembly), else null
    double* p_tmpE = nullptr;        // [E] staging of parameter uploads / gradient downloads
    int tape_every = 0;              // 0 = not recording
    int64_t tape_origin = 0;
    size_t n_ckpt = 0;
    std::vector<void*> ckpt;         // checkpoint k: the state at step tape_origin + k * tape_every
    void* ckpt_live = nullptr;       // the live state saved during rafem_adjoint
    size_t ckpt_bytes = 0;
    bool adj_ready = false;
    int seg_cap = 0;
    double *a_segT = nullptr, *a_segV = nullptr;   // [seg_cap + 1][N], [seg_cap][N]
    double *a_lam = nullptr, *a_mu = nullptr, *a_nu = nullptr, *a_h = nullptr, *a_dv = nullptr;
    double *a_ew4 = nullptr, *a_w = nullptr, *a_gs = nullptr, *a_gk = nullptr;
    double *a_mu1 = nullptr, *a_mu2 = nullptr, *a_nu1 = nullptr, *a_nu2 = nullptr;  // backward-sweep histories
    int32_t* a_count = nullptr;      // [iters_V, iters_T, adjoint status, recomputation status]
    // bounded device waits of the persistent solvers (rafem_set_wait_limit)
    long long wait_ns = kDefaultWaitNs;
    int wait_missing = 0;            // testing: grid-barrier arrivals the next solver launches start short of
};

namespace {

template <typename T>
cudaError_t dalloc(rafem_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T) + 64;  // slack for vector over-reads
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaMemsetAsync(q, 0, bytes, c->stream);
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return RAFEM_OK;
    if (e == cudaErrorMemoryAllocation) return RAFEM_ERR_OOM;
    return RAFEM_ERR_CUDA;
}

#define CK(expr)                                 \
    do {                                         \
        cudaError_t _e = (expr);                 \
        if (_e != cudaSuccess) return cuda_status(_e); \
    } while (0)

// Per-instance statistics of one solve (thread i handles instance i) and the step summary over instances
// (status: worst; iterations, refinements, relative residual: maximum).
__global__ void k_record(const InstState* inst, int n_inst, const GridBarrier* bar, int which, StatsDev* s,
                         rafem_step_stats* istats, int final_step) {
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        InstState st = inst[i];
        if (bar->err) st.status = bar->err;
        rafem_step_stats& q = istats[i];
        if (which == RAFEM_SYS_V) {
            q.iters_V += st.iters;
            q.refine_V += st.refine;
            q.relres_V = st.relres;
        } else {
            q.iters_T += st.iters;
            q.refine_T += st.refine;
            q.relres_T = st.relres;
        }
        const int status = st.status;
        if (status < 0 || q.status < 0)
            q.status = status < q.status ? status : q.status;
        else
            q.status = status > q.status ? status : q.status;
        if (final_step) q.step += 1;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    rafem_step_stats& c = s->cur;
    int iV = 0, iT = 0, rV = 0, rT = 0, stat = 0;
    double resV = 0.0, resT = 0.0;
    for (int i = 0; i < n_inst; ++i) {
        const rafem_step_stats& q = istats[i];
        iV = max(iV, q.iters_V);
        iT = max(iT, q.iters_T);
        rV = max(rV, q.refine_V);
        rT = max(rT, q.refine_T);
        resV = fmax(resV, q.relres_V);
        resT = fmax(resT, q.relres_T);
        if (q.status < 0 || stat < 0)
            stat = q.status < stat ? q.status : stat;
        else
            stat = q.status > stat ? q.status : stat;
    }
    c.iters_V = iV;
    c.iters_T = iT;
    c.refine_V = rV;
    c.refine_T = rT;
    c.relres_V = resV;
    c.relres_T = resT;
    c.status = stat;
    if (final_step) {
        c.step += 1;
        s->hist += 1;
        if (c.status < 0 || s->worst < 0)
            s->worst = c.status < s->worst ? c.status : s->worst;
        else
            s->worst = c.status > s->worst ? c.status : s->worst;
    }
}

__global__ void k_begin_step(StatsDev* s, rafem_step_stats* istats, int n_inst) {
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        rafem_step_stats& q = istats[i];
        const int64_t step = q.step;
        q = rafem_step_stats{};
        q.correctors = 1;
        q.step = step;
    }
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    rafem_step_stats& c = s->cur;
    c.status = 0;
    c.iters_V = c.iters_T = c.refine_V = c.refine_T = 0;
    c.correctors = 1;
    c.relres_V = c.relres_T = 0.0;
}

__global__ void k_set_step(StatsDev* s, long long step) {
    s->cur.step = step;
    s->worst = 0;
}

// Predictor: polynomial extrapolation in time of the free rows' solution from the last q + 1 solutions, used as
// the initial guess: linear 2 x^n - x^{n-1}, quadratic 3 x^n - 3 x^{n-1} + x^{n-2}, cubic
// 4 x^n - 6 x^{n-1} + 4 x^{n-2} - x^{n-3}, with q = min(order, hist - lag): after hist steps the temperature has
// hist + 1 states (T^0 included, lag 0) while the potential has been solved hist times (its initial field is not a
// solution, lag 1). The history shifts to keep the last `order` values.
__global__ void k_predict(int N, double* __restrict__ x, double* __restrict__ h1, double* __restrict__ h2,
                          double* __restrict__ h3, const uint8_t* __restrict__ bc, const StatsDev* s, int order,
                          int lag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double t = x[i];
    const double t1 = order >= 1 ? h1[i] : 0.0, t2 = order >= 2 ? h2[i] : 0.0, t3 = order >= 3 ? h3[i] : 0.0;
    const int q = min(order, s->hist - lag);
    if (!bc[i]) {
        if (q >= 3)
            x[i] = 4.0 * (t + t2) - 6.0 * t1 - t3;
        else if (q == 2)
            x[i] = 3.0 * (t - t1) + t2;
        else if (q == 1)
            x[i] = 2.0 * t - t1;
    }
    if (order >= 3) h3[i] = t2;
    if (order >= 2) h2[i] = t1;
    if (order >= 1) h1[i] = t;
}

__global__ void k_reset_hist(StatsDev* s) { s->hist = 0; }

__global__ void k_corr_init(CorrDev* c) {
    c->pass = 0;
    c->converged = 0;
    c->change = 0.0;
    c->newton_rr = 0.0;
}

// After a corrector pass: count it, read max |T^{k+1} - T^k| (non-negative double stored as its bit pattern) and
// decide whether another pass follows; with a graph the decision drives the conditional WHILE node.
__global__ void k_corr_check(CorrDev* c, const double* scratch, double tol, int max_pass,
                             cudaGraphConditionalHandle h, int use_handle) {
    const double change = *scratch;
    c->pass += 1;
    c->change = change;
    c->converged = change < tol;
    const int more = !(change < tol) && c->pass < max_pass && change == change;
    if (use_handle) cudaGraphSetConditional(h, more ? 1u : 0u);
}

// End of a corrector step: pass count into the statistics, step counters advanced; a step whose passes did not
// converge reports RAFEM_NOT_CONVERGED unless a worse status was recorded.
__global__ void k_corr_finish(StatsDev* s, rafem_step_stats* istats, int n_inst, const CorrDev* c) {
    const int st_add = c->converged ? RAFEM_OK : RAFEM_NOT_CONVERGED;
    for (int i = threadIdx.x; i < n_inst; i += blockDim.x) {
        rafem_step_stats& q = istats[i];
        q.correctors = c->pass;
        q.step += 1;
        if (q.status >= 0 && st_add > q.status) q.status = st_add;
    }
    if (threadIdx.x != 0) return;
    rafem_step_stats& cur = s->cur;
    cur.correctors = c->pass;
    if (cur.status >= 0 && st_add > cur.status) cur.status = st_add;
    cur.step += 1;
    s->hist += 1;
    if (cur.status < 0 || s->worst < 0)
        s->worst = cur.status < s->worst ? cur.status : s->worst;
    else
        s->worst = cur.status > s->worst ? cur.status : s->worst;
}

__global__ void k_jacobi_apply(int N, const int32_t* __restrict__ diag, const double* __restrict__ A,
                               const double* __restrict__ r, double* __restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) z[i] = r[i] / A[diag[i]];
}

__global__ void k_fold_worst(const StatsDev* s, int32_t* acc) {
    const int w = s->worst, a = *acc;
    *acc = (w < 0 || a < 0) ? min(w, a) : max(w, a);
}

__global__ void k_init_fields(int N, double T0, const uint8_t* bcT, const double* gT, const uint8_t* bcV,
                              const double* gV, double* T, double* V) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T[i] = bcT[i] ? gT[i] : T0;
    V[i] = bcV[i] ? gV[i] : 0.0;
}

SolveArgs make_args(rafem_ctx* c, int which, const double* b, double* x) {
    SolveArgs a{};
    a.N = c->N;
    a.rp = c->rp;
    a.ci = c->ci;
    a.ci16 = c->ci16;
    a.pat_off = c->pat_off;
    a.pat_pool = c->pat_pool;
    a.A = which == RAFEM_SYS_V ? c->valsV : c->valsT;
    a.A32 = which == RAFEM_SYS_V ? c->valsV32 : c->valsT32;
    a.diag = c->diag;
    a.b = b;
    a.x = x;
    a.r = c->wr; a.u = c->wu; a.w = c->ww; a.p = c->wp; a.s = c->ws; a.dinv = c->wdinv;
    a.r32 = c->fr; a.u32 = c->fu; a.w32 = c->fw; a.p32 = c->fp; a.s32 = c->fs; a.d32 = c->fd; a.dinv32 = c->fdinv;
    a.z = c->pz; a.q = c->pq; a.ma = c->pm0; a.mb = c->pm1;
    a.n_tiles = c->n_tiles;
    a.tile_r0 = c->tile_r0;
    a.tile_r1 = c->tile_r1;
    a.tile_inst = c->tile_inst;
    a.n_inst = c->n_inst;
    a.inst_t0 = c->inst_t0;
    a.inst_t1 = c->inst_t1;
    a.inst = which == RAFEM_SYS_V ? c->instV : c->instT;
    a.partial = c->partial;
    a.bar = c->bar;
    a.tol = c->prm.tol;
    a.inner_tol = c->prm.inner_tol;
    a.max_iter = c->prm.max_iter;
    a.max_refine = c->prm.max_refine;
    a.spin_limit_ns = c->wait_ns;
    a.bar_missing = c->wait_missing;
    return a;
}

cudaError_t enqueue_assemble_raw(rafem_ctx* c, int which, const double* T_sigma, const double* T_old, bool with_y);

// ILU(0) factors of system `which` after its matrix changed: the combined layout, then the ring solver's copies.
cudaError_t ilu_refactor(rafem_ctx* c, int which, cudaStream_t st) {
    const bool V = which == RAFEM_SYS_V;
    double* Ap = V ? c->ilu_AV : c->ilu_AT;
    double* F = V ? c->ilu_FV : c->ilu_FT;
    double* D = V ? c->ilu_DV : c->ilu_DT;
    const cudaError_t e = launch_ilu_refactor(c->il, V ? c->valsV : c->valsT, Ap, F, D, st);
    if (e != cudaSuccess) return e;
    return launch_ilu_ring_split(c->ir[V ? 0 : 1], Ap, F, D, c->prm.precision == RAFEM_PRECISION_MIXED, st);
}

// Assembly of one system; with ILU(0) the potential matrix is refactored right after it is assembled. with_y: the
// potential's assembly also computes the projection predictor's Y = A D (double-word gather, basis of 4, basis
// already built).
cudaError_t enqueue_assemble(rafem_ctx* c, int which, const double* T_sigma, const double* T_old,
                             bool with_y = false) {
    cudaError_t e = enqueue_assemble_raw(c, which, T_sigma, T_old, with_y);
    if (e != cudaSuccess || !c->ilu || which != RAFEM_SYS_V) return e;
    return ilu_refactor(c, RAFEM_SYS_V, c->stream);
}

cudaError_t enqueue_assemble_raw(rafem_ctx* c, int which, const double* T_sigma, const double* T_old, bool with_y) {
    cudaError_t e;
    if (c->dw) {
        float* v32 = c->valsV32;  // FP32 copy, when the context keeps one
        if (which == RAFEM_SYS_V)
            return launch_assemble_V_gather_dw(c->gd, c->gdw, c->N, c->rp, c->ci, c->diag, c->el, T_sigma,
                                               c->prm.alpha_sigma, c->bcV, c->gV, c->valsV, v32, c->bV, c->prm.lift,
                                               with_y ? c->proj_D : nullptr, with_y ? c->proj_Y : nullptr,
                                               with_y ? c->proj_kin : nullptr, c->stream);
        return launch_rhs_T_gather_dw(c->gd, c->gdw, c->N, c->el, T_sigma, T_old, c->V, c->bcT, c->gT, c->bTc,
                                      c->prm.alpha_sigma, c->bT, c->stream);
    }
    if (c->gather) {
        float* v32 = c->valsV32;  // FP32 copy, when the context keeps one
        if (which == RAFEM_SYS_V)
            return launch_assemble_V_gather(c->gd, c->N, c->rp, c->ci, c->diag, c->el, T_sigma, c->prm.alpha_sigma,
                                            c->bcV, c->gV, c->valsV, v32, c->bV, c->prm.lift, c->stream);
        return launch_rhs_T_gather(c->gd, c->N, c->el, T_sigma, T_old, c->V, c->bcT, c->gT, c->bTc,
                                   c->prm.alpha_sigma, c->prm.rho_c / c->prm.dt, c->bT, c->stream);
    }
    if (which == RAFEM_SYS_V) {
        e = launch_init_rhs(c->N, c->bcV, c->gV, nullptr, c->bV, c->stream);
        if (e != cudaSuccess) return e;
        float* v32 = c->valsV32;  // FP32 copy, when the context keeps one
        for (int col = 0; col < c->n_colors; ++col) {
            e = launch_assemble_V(c->el, c->color_off[col], c->color_off[col + 1], T_sigma, c->bcV, c->gV,
                                  c->prm.alpha_sigma, c->valsV, v32, c->bV, c->prm.lift, c->stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    e = launch_init_rhs(c->N, c->bcT, c->gT, c->bTc, c->bT, c->stream);
    if (e != cudaSuccess) return e;
    for (int col = 0; col < c->n_colors; ++col) {
        e = launch_rhs_T(c->el, c->color_off[col], c->color_off[col + 1], T_sigma, T_old, c->V, c->bcT,
                         c->prm.alpha_sigma, c->prm.rho_c / c->prm.dt, c->bT, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The potential's initial guess comes from the projection predictor (it needs A SPD: the symmetric lift, any
// solver).
bool projected_V(const rafem_ctx* c) {
    return c->prm.predictor == RAFEM_PREDICT_PROJECT && c->prm.lift == RAFEM_LIFT_SYMMETRIC;
}

// The projection's Y = A D comes from the potential's assembly: double-word gather assembly, basis of up to 4.
bool fused_V(const rafem_ctx* c) { return c->dw && projected_V(c) && c->proj_D && proj_stride(c->proj_k) == 4; }

ProjArgs proj_args(const rafem_ctx* c) {
    ProjArgs a{};
    a.n_tiles = c->n_tiles;
    a.n_sub = c->proj_sub;
    a.dw = c->dw ? 1 : 0;
    a.tile_r0 = c->tile_r0;
    a.tile_r1 = c->tile_r1;
    a.tile_inst = c->tile_inst;
    a.n_inst = c->n_inst;
    a.inst_t0 = c->inst_t0;
    a.inst_t1 = c->inst_t1;
    a.sell = c->sell ? 1 : 0;
    a.rp = c->rp;
    a.ci = c->ci;
    a.ci16 = c->ci16;
    a.A = c->valsV;
    a.bc = c->bcV;
    a.b = c->bV;
    a.x = c->V;
    a.kmax = c->proj_k;
    a.partial = c->proj_partial;
    a.coef = c->proj_coef;
    a.kin = c->proj_kin;
    a.kout = c->proj_kout;
    a.D = c->proj_D;
    a.Y = c->proj_Y;
    a.r0 = c->proj_r0;
    return a;
}

// The step's potential assembly. fuse (fused_V, and V is final when it runs): the projection basis is built from
// the previous solution first, and the assembly accumulates Y = A D along with the matrix.
cudaError_t enqueue_assemble_V_step(rafem_ctx* c, bool fuse) {
    if (fuse) {
        const cudaError_t e = launch_projection_basis(proj_args(c), &c->stats->hist, 1, c->stream);
        if (e != cudaSuccess) return e;
    }
    return enqueue_assemble(c, RAFEM_SYS_V, c->T, c->T, fuse);
}

cudaError_t enqueue_solve(rafem_ctx* c, int which, const double* b, double* x) {
    // the residual of the projected guess serves only the potential solve enqueued right after the projection
    const bool r0_fresh = c->r0_fresh && which == RAFEM_SYS_V && b == c->bV && x == c->V;
    if (which == RAFEM_SYS_V) c->r0_fresh = false;
    if (c->ilu) {
        IluRingSolve s{};
        s.d = &c->ir[which == RAFEM_SYS_V ? 0 : 1];
        s.mixed = c->prm.precision == RAFEM_PRECISION_MIXED;
        s.N = c->N;
        s.dinv64 = which == RAFEM_SYS_V ? c->ilu_DV : c->ilu_DT;
        s.b = b;
        s.x = x;
        s.bar = c->bar;
        s.inst = which == RAFEM_SYS_V ? c->instV : c->instT;
        s.tol = c->prm.tol;
        s.inner_tol = c->prm.inner_tol;
        s.max_iter = c->prm.max_iter;
        s.max_refine = c->prm.max_refine;
        s.spin_limit_ns = c->wait_ns;
        s.bar_missing = c->wait_missing;
        return launch_ilu_ring(s, c->ir_grid, c->stream);
    }
    if (c->prm.solver == RAFEM_SOLVER_GMRES) {
        GmresArgs g{};
        g.N = c->N;
        g.m = c->gm_m;
        g.m_min = c->prm.gmres_min_restart;
        g.sp = c->rp;
        g.sc = c->ci;
        g.sc16 = c->ci16;
        g.pat_off = c->pat_off;
        g.pat_pool = c->pat_pool;
        g.A = which == RAFEM_SYS_V ? c->valsV : c->valsT;
        g.diag = c->diag;
        g.b = b;
        g.x = x;
        g.ld = c->gm_ld;
        g.V = c->gm_V;
        g.w0 = c->gm_w0;
        g.w1 = c->gm_w1;
        g.z = c->gm_z;
        g.dinv = c->gm_dinv;
        g.H = c->gm_H;
        g.partial = c->gm_partial;
        g.bar = c->bar;
        g.inst = which == RAFEM_SYS_V ? c->instV : c->instT;
        g.tol = c->prm.tol;
        g.max_iter = c->prm.max_iter;
        g.spin_limit_ns = c->wait_ns;
        g.bar_missing = c->wait_missing;
        return launch_gmres(g, c->gm_grid, c->stream);
    }
    if (c->prm.solver == RAFEM_SOLVER_BICGSTAB) {
        BicgArgs g{};
        g.N = c->N;
        g.sp = c->rp;
        g.sc = c->ci;
        g.sc16 = c->ci16;
        g.pat_off = c->pat_off;
        g.pat_pool = c->pat_pool;
        g.A = which == RAFEM_SYS_V ? c->valsV : c->valsT;
        g.diag = c->diag;
        g.b = b;
        g.x = x;
        g.r = c->bg_r;
        g.rh = c->bg_rh;
        g.p = c->bg_p;
        g.ph = c->bg_ph;
        g.v = c->bg_v;
        g.s = c->bg_s;
        g.sh = c->bg_sh;
        g.t = c->bg_t;
        g.dinv = c->bg_dinv;
        g.partial = c->bg_partial;
        g.bar = c->bar;
        g.inst = which == RAFEM_SYS_V ? c->instV : c->instT;
        g.tol = c->prm.tol;
        g.max_iter = c->prm.max_iter;
        g.spin_limit_ns = c->wait_ns;
        g.bar_missing = c->wait_missing;
        return launch_bicgstab(g, c->bg_grid, c->stream);
    }
    SolveArgs a = make_args(c, which, b, x);
    if (r0_fresh) {
        // the projection predictor left the residual of its guess: no first residual SpMV
        a.r0 = c->proj_r0;
        a.r0_ok = c->proj_kout;
    }
    return launch_krylov(a, c->lanes, c->prm.precision, c->prm.solver == RAFEM_SOLVER_PIPECG, c->grid, c->block,
                         c->stream);
}

// Initial guess of a step's solve (the predictor of Sec. II-A's predictor-corrector loop): polynomial
// extrapolation of order 1..3, or (predictor 4) for the potential the A-orthogonal projection onto its last
// proj_basis solutions, which needs an SPD system (the symmetric lift, any solver; order 2 otherwise, and for the
// thermal system, whose few iterations would not repay the extra pass).
// fused: the basis and Y were made with the assembly (enqueue_assemble_V_step).
cudaError_t enqueue_predict(rafem_ctx* c, int which, bool fused = false) {
    if (!c->prm.predictor) return cudaSuccess;
    const bool V = which == RAFEM_SYS_V;
    if (V && projected_V(c)) {
        c->r0_fresh = true;
        return fused ? launch_projection_rest(proj_args(c), false, c->stream)
                     : launch_projection(proj_args(c), &c->stats->hist, 1, c->stream);
    }
    const int order = c->prm.predictor == RAFEM_PREDICT_PROJECT ? 2 : c->prm.predictor;
    if (V)
        k_predict<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->N, c->V, c->V_hist, c->V_hist2, c->V_hist3, c->bcV,
                                                             c->stats, order, 1);
    else
        k_predict<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->N, c->T, c->T_hist, c->T_hist2, c->T_hist3, c->bcT,
                                                             c->stats, order, 0);
    return cudaGetLastError();
}

// Host buffers of a host-state step (any may be null): state in before the step, fields out after it.
struct StepIO {
    const double *T_in, *V_in;
    double *T_out, *V_out;
};

// One lagged pass: sigma and the mass term both use the current T. With io, the step also moves its state to
// and from host memory: T in first on the step's stream (the potential assembly reads it), V in on the second
// stream while the potential is assembled (only its predictor reads V), V out on the second stream as soon as
// the potential is solved (during the thermal half of the step), T out at the end; the second stream joins
// before the step ends.
cudaError_t enqueue_step_io(rafem_ctx* c, const StepIO* io) {
    cudaError_t e;
    cudaStream_t S = c->stream, I = c->io_stream;
    const size_t nb = (size_t)c->N * sizeof(double);
    const bool vin = io && io->V_in, vout = io && io->V_out;
    c->r0_fresh = false;
    if (io && io->T_in && (e = cudaMemcpyAsync(c->T, io->T_in, nb, cudaMemcpyHostToDevice, S)) != cudaSuccess) return e;
    if (vin) {
        if ((e = cudaEventRecord(c->io_ev[0], S)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(I, c->io_ev[0], 0)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(c->V, io->V_in, nb, cudaMemcpyHostToDevice, I)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(c->io_ev[1], I)) != cudaSuccess) return e;
    }
    k_begin_step<<<1, 128, 0, S>>>(c->stats, c->istats, c->n_inst);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool fuse = fused_V(c) && !vin;  // the fused basis would have to wait for V before the assembly
    if ((e = enqueue_assemble_V_step(c, fuse)) != cudaSuccess) return e;
    if (vin && (e = cudaStreamWaitEvent(S, c->io_ev[1], 0)) != cudaSuccess) return e;
    if ((e = enqueue_predict(c, RAFEM_SYS_V, fuse)) != cudaSuccess) return e;
    if ((e = enqueue_solve(c, RAFEM_SYS_V, c->bV, c->V)) != cudaSuccess) return e;
    k_record<<<1, 128, 0, S>>>(c->instV, c->n_inst, c->bar, RAFEM_SYS_V, c->stats, c->istats, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (vout) {
        if ((e = cudaEventRecord(c->io_ev[2], S)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(I, c->io_ev[2], 0)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(io->V_out, c->V, nb, cudaMemcpyDeviceToHost, I)) != cudaSuccess) return e;
    }
    if (vin || vout) {
        if ((e = cudaEventRecord(c->io_ev[3], I)) != cudaSuccess) return e;
    }
    if ((e = enqueue_assemble(c, RAFEM_SYS_T, c->T, c->T)) != cudaSuccess) return e;
    if ((e = enqueue_predict(c, RAFEM_SYS_T)) != cudaSuccess) return e;
    if ((e = enqueue_solve(c, RAFEM_SYS_T, c->bT, c->T)) != cudaSuccess) return e;
    k_record<<<1, 128, 0, S>>>(c->instT, c->n_inst, c->bar, RAFEM_SYS_T, c->stats, c->istats, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (io && io->T_out && (e = cudaMemcpyAsync(io->T_out, c->T, nb, cudaMemcpyDeviceToHost, S)) != cudaSuccess)
        return e;
    if ((vin || vout) && (e = cudaStreamWaitEvent(S, c->io_ev[3], 0)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t enqueue_step(rafem_ctx* c) { return enqueue_step_io(c, nullptr); }

// Traced step: the same launches as enqueue_step with an event between regions (Assembly, Predict, Solve).
cudaError_t enqueue_step_traced(rafem_ctx* c) {
    cudaError_t e;
    for (int i = 0; i < 8; ++i)
        if (!c->ev[i] && (e = cudaEventCreate(&c->ev[i])) != cudaSuccess) return e;
    k_begin_step<<<1, 128, 0, c->stream>>>(c->stats, c->istats, c->n_inst);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    nvtxRangePushA("Assembly");
    cudaEventRecord(c->ev[0], c->stream);
    if ((e = enqueue_assemble_V_step(c, fused_V(c))) != cudaSuccess) return e;
    cudaEventRecord(c->ev[1], c->stream);
    nvtxRangePop();
    nvtxRangePushA("Predict");
    if ((e = enqueue_predict(c, RAFEM_SYS_V, fused_V(c))) != cudaSuccess) return e;
    cudaEventRecord(c->ev[6], c->stream);
    nvtxRangePop();
    nvtxRangePushA("Solve");
    if ((e = enqueue_solve(c, RAFEM_SYS_V, c->bV, c->V)) != cudaSuccess) return e;
    cudaEventRecord(c->ev[2], c->stream);
    nvtxRangePop();
    k_record<<<1, 128, 0, c->stream>>>(c->instV, c->n_inst, c->bar, RAFEM_SYS_V, c->stats, c->istats, 0);
    nvtxRangePushA("Assembly");
    cudaEventRecord(c->ev[3], c->stream);
    if ((e = enqueue_assemble(c, RAFEM_SYS_T, c->T, c->T)) != cudaSuccess) return e;
    cudaEventRecord(c->ev[4], c->stream);
    nvtxRangePop();
    nvtxRangePushA("Predict");
    if ((e = enqueue_predict(c, RAFEM_SYS_T)) != cudaSuccess) return e;
    cudaEventRecord(c->ev[7], c->stream);
    nvtxRangePop();
    nvtxRangePushA("Solve");
    if ((e = enqueue_solve(c, RAFEM_SYS_T, c->bT, c->T)) != cudaSuccess) return e;
    cudaEventRecord(c->ev[5], c->stream);
    nvtxRangePop();
    k_record<<<1, 128, 0, c->stream>>>(c->instT, c->n_inst, c->bar, RAFEM_SYS_T, c->stats, c->istats, 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    float ms[6];
    cudaEventElapsedTime(&ms[0], c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&ms[1], c->ev[6], c->ev[2]);
    cudaEventElapsedTime(&ms[2], c->ev[3], c->ev[4]);
    cudaEventElapsedTime(&ms[3], c->ev[7], c->ev[5]);
    cudaEventElapsedTime(&ms[4], c->ev[1], c->ev[6]);
    cudaEventElapsedTime(&ms[5], c->ev[4], c->ev[7]);
    c->trace.ms_assemble_V += ms[0];
    c->trace.ms_solve_V += ms[1];
    c->trace.ms_assemble_T += ms[2];
    c->trace.ms_solve_T += ms[3];
    c->trace.ms_predict_V += ms[4];
    c->trace.ms_predict_T += ms[5];
    c->trace.steps += 1;
    c->trace.solves += 1;
    std::vector<InstState> iv(c->n_inst), it(c->n_inst);
    if ((e = cudaMemcpy(iv.data(), c->instV, c->n_inst * sizeof(InstState), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpy(it.data(), c->instT, c->n_inst * sizeof(InstState), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    int mv = 0, mt = 0, mr = 0;
    for (int i = 0; i < c->n_inst; ++i) {
        mv = std::max(mv, iv[i].iters);
        mt = std::max(mt, it[i].iters);
        mr = std::max(mr, iv[i].refine);
    }
    c->trace.iters_V += mv;
    c->trace.iters_T += mt;
    c->trace.refine_V += mr;
    return cudaSuccess;
}

// ---- corrector passes on the device --------------------------------------------------------------------------
// Prologue: T_old = T (the mass term keeps T^n), statistics and pass counter cleared.
// Monolithic step: Newton starts from the lagged staggered step (V, then T, each an SPD solve with sigma(T^n)),
// which differs from the coupled solution only through the step's own temperature change, so the first Newton
// residual is already small. The start's own solves are not counted in the step statistics.
cudaError_t enqueue_corr_prologue(rafem_ctx* c) {
    cudaError_t e = cudaMemcpyAsync(c->T_old, c->T, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
    k_begin_step<<<1, 128, 0, c->stream>>>(c->stats, c->istats, c->n_inst);
    k_corr_init<<<1, 1, 0, c->stream>>>(c->corr);
    if ((e = cudaGetLastError()) != cudaSuccess || !c->mono) return e;
    c->r0_fresh = false;
    if ((e = enqueue_assemble(c, RAFEM_SYS_V, c->T, c->T)) != cudaSuccess) return e;
    if ((e = enqueue_solve(c, RAFEM_SYS_V, c->bV, c->V)) != cudaSuccess) return e;
    if ((e = enqueue_assemble(c, RAFEM_SYS_T, c->T, c->T_old)) != cudaSuccess) return e;
    return enqueue_solve(c, RAFEM_SYS_T, c->bT, c->T);
}

// The coupled Jacobian (2 x 2 blocks on the node pattern) and residual at the current (V, T): by rows on the
// gather lists when the context has them, else by the colour scatter followed by the Dirichlet rows.
cudaError_t enqueue_coupled_assembly(rafem_ctx* c) {
    cudaStream_t st = c->stream;
    const int N = c->N;
    const double c_dt = c->prm.rho_c / c->prm.dt;
    if (c->mg.cab)
        return launch_coupled_gather(c->mg, c->gd, N, c->rp, c->ci, c->diag, c->el, c->V, c->T, c->T_old, c->prm.alpha_sigma,
                                     c_dt, c->prm.perf, c->prm.T_a, c->bcV, c->bcT, c->gV, c->gT, c->m_vals4, c->m_R,
                                     st);
    cudaError_t e = cudaMemsetAsync(c->m_R, 0, 2 * (size_t)N * sizeof(double), st);
    if (e != cudaSuccess) return e;
    for (int q = 0; q < c->n_colors; ++q) {
        e = launch_coupled(c->el, c->color_off[q], c->color_off[q + 1], c->e_clist, c->V, c->T, c->T_old,
                           c->prm.alpha_sigma, c_dt, c->prm.perf, c->prm.T_a, c->m_vals4, c->m_R, st);
        if (e != cudaSuccess) return e;
    }
    return launch_coupled_dirichlet(N, c->sell ? 1 : 0, c->rp, c->diag, c->bcV, c->bcT, c->gV, c->gT, c->V, c->T,
                                    c->m_vals4, c->m_R, st);
}

// The Newton linear solve J delta = R by flexible GMRES with the split-system preconditioner (mono_fgmres.cu): a
// fixed sequence of kFgMax outer iterations whose launches return at once after convergence, then delta and
// (V, T) -= delta. The inner solves are mixed-precision Jacobi-PCG launches (FP32 iterations, FP64 residual) on
// the assembled split matrices (A_V with sigma at T^n from the step's staggered start, the constant A_T), each to
// a relative residual of kFgInnerTol.
// Looser inner solves trade inner iterations for outer ones: of 0.05 to 0.6, 0.4 was the fastest at 127^3.
constexpr double kFgInnerTol = 0.4;
cudaError_t enqueue_newton_fgmres(rafem_ctx* c) {
    cudaStream_t st = c->stream;
    const int N = c->N, n2 = 2 * N, G = c->fg_G;
    const size_t ld = c->fg_ld;
    FgState* fs = c->fg_st;
    cudaError_t e = cudaMemsetAsync(&fs->done, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if ((e = launch_fg_dots(n2, c->m_R, c->fg_V, ld, 0, fs, c->fg_partial, G, st)) != cudaSuccess) return e;
    if ((e = launch_fg_init(fs, c->fg_partial, G, &c->corr->newton_rr, c->prm.tol, st)) != cudaSuccess) return e;
    if ((e = launch_fg_scale(n2, c->m_R, c->fg_V, fs, st)) != cudaSuccess) return e;
    for (int j = 0; j < kFgMax; ++j) {
        const double* Vj = c->fg_V + (size_t)j * ld;
        if ((e = launch_fg_split(N, Vj, c->fg_rV, c->fg_rT, c->fg_zV, c->fg_zT, fs, st)) != cudaSuccess) return e;
        for (int which : {RAFEM_SYS_V, RAFEM_SYS_T}) {
            const bool V = which == RAFEM_SYS_V;
            if (!V && (e = launch_fg_couple(N, c->rp, c->ci, c->ci16, c->m_vals4, c->fg_zV, c->fg_rT, fs, st)) !=
                          cudaSuccess)
                return e;
            SolveArgs a = make_args(c, which, V ? c->fg_rV : c->fg_rT, V ? c->fg_zV : c->fg_zT);
            a.tol = kFgInnerTol;
            a.skip = &fs->done;
            a.r0 = a.b;  // x0 = 0: the starting residual is the right-hand side (no first SpMV)
            a.r0_ok = c->fg_one;
            if ((e = launch_krylov(a, c->lanes, c->valsV32 ? RAFEM_PRECISION_MIXED : RAFEM_PRECISION_FP64, false,
                                   c->grid, c->block, st)) != cudaSuccess)
                return e;
            if ((e = launch_fg_count(fs, V ? c->instV : c->instT, which, st)) != cudaSuccess) return e;
        }
        double* Zj = c->fg_Z + (size_t)j * ld;
        if ((e = launch_fg_spmv(N, c->rp, c->ci, c->ci16, c->m_vals4, c->fg_zV, c->fg_zT, c->fg_w, Zj, fs, st)) !=
            cudaSuccess)
            return e;
        // Gram-Schmidt: the second pass's launches return at once when the first pass was enough
        for (int pass = 1; pass <= 2; ++pass) {
            if ((e = launch_fg_dots(n2, c->fg_w, c->fg_V, ld, j + 1, fs, c->fg_partial, G, st, pass)) != cudaSuccess)
                return e;
            if ((e = launch_fg_gs(fs, c->fg_partial, G, j, pass, st)) != cudaSuccess) return e;
            if ((e = launch_fg_sub(n2, c->fg_w, c->fg_V, ld, j, fs, c->fg_V + (size_t)(j + 1) * ld, pass, st)) !=
                cudaSuccess)
                return e;
        }
    }
    if ((e = launch_fg_finish(n2, c->fg_Z, ld, fs, c->m_D, c->instV, c->instT, st)) != cudaSuccess) return e;
    k_record<<<1, 128, 0, st>>>(c->instV, c->n_inst, c->bar, RAFEM_SYS_V, c->stats, c->istats, 0);
    k_record<<<1, 128, 0, st>>>(c->instT, c->n_inst, c->bar, RAFEM_SYS_T, c->stats, c->istats, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_newton_update(N, c->m_D, c->V, c->T, st);
}

// One Newton iteration of the monolithic coupled step: assemble the 2N x 2N Jacobian and residual at the current
// (V, T), solve J delta = R with block-Jacobi BiCGSTAB, (V, T) -= delta.
cudaError_t enqueue_newton(rafem_ctx* c) {
    cudaStream_t st = c->stream;
    const int N = c->N;
    cudaError_t e = enqueue_coupled_assembly(c);
    if (e != cudaSuccess) return e;
    if (c->fg_st) return enqueue_newton_fgmres(c);
    if ((e = cudaMemsetAsync(c->m_D, 0, 2 * (size_t)N * sizeof(double), st)) != cudaSuccess) return e;
    BicgArgs g{};
    g.block = 2;
    g.N = N;
    g.sp = c->rp;
    g.sc = c->ci;
    g.sc16 = c->ci16;
    g.A = c->m_vals4;
    g.diag = c->diag;
    g.b = c->m_R;
    g.x = c->m_D;
    g.r = c->mb_r;
    g.rh = c->mb_rh;
    g.p = c->mb_p;
    g.ph = c->mb_ph;
    g.v = c->mb_v;
    g.s = c->mb_s;
    g.sh = c->mb_sh;
    g.t = c->mb_t;
    g.dinv = c->mb_dinv;
    g.partial = c->mb_partial;
    g.bar = c->bar;
    g.inst = c->instV;
    g.tol = c->prm.tol;
    g.max_iter = c->prm.max_iter;
    g.spin_limit_ns = c->wait_ns;
    g.bar_missing = c->wait_missing;
    g.newton = &c->corr->newton_rr;  // inexact Newton: each linear solve only as accurate as the iteration needs
    if ((e = launch_bicgstab(g, c->mb_grid, st)) != cudaSuccess) return e;
    k_record<<<1, 128, 0, st>>>(c->instV, c->n_inst, c->bar, RAFEM_SYS_V, c->stats, c->istats, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_newton_update(N, c->m_D, c->V, c->T, st);
}

// One corrector pass (sigma at the newest temperature iterate T, mass term at T_old), or one Newton iteration of
// the monolithic step, then the convergence test on max |T^{k+1} - T^k|.
cudaError_t enqueue_corrector_pass(rafem_ctx* c, cudaGraphConditionalHandle h, int use_handle) {
    cudaError_t e = cudaMemcpyAsync(c->T_prev, c->T, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
    if (c->mono) {
        if ((e = enqueue_newton(c)) != cudaSuccess) return e;
        if ((e = launch_max_abs_diff(c->N, c->T, c->T_prev, c->scratch, c->stream)) != cudaSuccess) return e;
        k_corr_check<<<1, 1, 0, c->stream>>>(c->corr, c->scratch, c->prm.corrector_tol, c->prm.n_corrector, h,
                                            use_handle);
        return cudaGetLastError();
    }
    if ((e = enqueue_assemble(c, RAFEM_SYS_V, c->T, c->T_old)) != cudaSuccess) return e;
    if ((e = enqueue_solve(c, RAFEM_SYS_V, c->bV, c->V)) != cudaSuccess) return e;
    k_record<<<1, 128, 0, c->stream>>>(c->instV, c->n_inst, c->bar, RAFEM_SYS_V, c->stats, c->istats, 0);
    if ((e = enqueue_assemble(c, RAFEM_SYS_T, c->T, c->T_old)) != cudaSuccess) return e;
    if ((e = enqueue_solve(c, RAFEM_SYS_T, c->bT, c->T)) != cudaSuccess) return e;
    k_record<<<1, 128, 0, c->stream>>>(c->instT, c->n_inst, c->bar, RAFEM_SYS_T, c->stats, c->istats, 0);
    if ((e = launch_max_abs_diff(c->N, c->T, c->T_prev, c->scratch, c->stream)) != cudaSuccess) return e;
    k_corr_check<<<1, 1, 0, c->stream>>>(c->corr, c->scratch, c->prm.corrector_tol, c->prm.n_corrector, h,
                                        use_handle);
    return cudaGetLastError();
}

cudaError_t enqueue_corr_epilogue(rafem_ctx* c) {
    k_corr_finish<<<1, 128, 0, c->stream>>>(c->stats, c->istats, c->n_inst, c->corr);
    return cudaGetLastError();
}

// The corrector step as one graph: prologue -> WHILE(more passes) { pass } -> epilogue. The body's last kernel
// sets the loop condition, so a step needs no host round trip. If the graph cannot be built, steps fall back to
// a host loop over the same launches (one small read-back per pass).
void ensure_corr_graph(rafem_ctx* c) {
    if (c->corr_graph || c->corr_graph_failed) return;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
    cudaGraph_t g = nullptr;
    bool ok = false;
    do {
        if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
        cudaGraph_t out = nullptr;
        if (cudaStreamBeginCaptureToGraph(c->stream, g, nullptr, nullptr, 0, mode) != cudaSuccess) break;
        cudaError_t e1 = enqueue_corr_prologue(c);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &out);
        if (e1 != cudaSuccess || e2 != cudaSuccess) break;
        size_t n = 0;
        if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) break;
        std::vector<cudaGraphNode_t> nodes(n), sinks;
        if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) break;
        for (cudaGraphNode_t nd : nodes) {
            size_t k = 0;
            if (cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &k) == cudaSuccess && k == 0) sinks.push_back(nd);
        }
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t loop;
        if (cudaGraphAddNode(&loop, g, sinks.data(), nullptr, sinks.size(), &cp) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, mode) != cudaSuccess) break;
        e1 = enqueue_corrector_pass(c, h, 1);
        e2 = cudaStreamEndCapture(c->stream, &out);
        if (e1 != cudaSuccess || e2 != cudaSuccess) break;
        if (cudaStreamBeginCaptureToGraph(c->stream, g, &loop, nullptr, 1, mode) != cudaSuccess) break;
        e1 = enqueue_corr_epilogue(c);
        e2 = cudaStreamEndCapture(c->stream, &out);
        if (e1 != cudaSuccess || e2 != cudaSuccess) break;
        if (cudaGraphInstantiate(&c->corr_graph, g, 0) != cudaSuccess) {
            c->corr_graph = nullptr;
            break;
        }
        ok = true;
    } while (false);
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        c->corr_graph_failed = true;
        cudaGetLastError();
    }
}

// One corrector step: the conditional graph, or the host loop when the graph is not available.
cudaError_t launch_corrector_step(rafem_ctx* c) {
    if (!c->tracing) {
        ensure_corr_graph(c);
        if (c->corr_graph) return cudaGraphLaunch(c->corr_graph, c->stream);
    }
    cudaError_t e = enqueue_corr_prologue(c);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < c->prm.n_corrector; ++pass) {
        if ((e = enqueue_corrector_pass(c, 0, 0)) != cudaSuccess) return e;
        CorrDev h;
        if ((e = cudaMemcpyAsync(&h, c->corr, sizeof(h), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
        if (h.converged || !(h.change == h.change)) break;
    }
    return enqueue_corr_epilogue(c);
}

void drop_graphs(rafem_ctx* c) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->corr_graph) cudaGraphExecDestroy(c->corr_graph);
    if (c->io_graph) cudaGraphExecDestroy(c->io_graph);
    c->graph = nullptr;
    c->corr_graph = nullptr;
    c->io_graph = nullptr;
    c->graph_failed = false;
    c->corr_graph_failed = false;
    c->io_graph_failed = false;
}

// The step graph (captured once; direct launches if capture is not possible).
void ensure_graph(rafem_ctx* c) {
    if (c->graph || c->graph_failed) return;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e1 = enqueue_step(c);
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (e1 == cudaSuccess && e2 == cudaSuccess && g) {
            if (cudaGraphInstantiate(&c->graph, g, 0) != cudaSuccess) c->graph = nullptr;
            size_t n = 0;
            c->graph_kernels = 0;
            if (c->graph && cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess && n > 0) {
                std::vector<cudaGraphNode_t> nodes(n);
                if (cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess)
                    for (size_t q = 0; q < n; ++q) {
                        cudaGraphNodeType t;
                        if (cudaGraphNodeGetType(nodes[q], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
                            c->graph_kernels += 1;
                    }
            }
        }
        if (g) cudaGraphDestroy(g);
    }
    if (!c->graph) {
        c->graph_failed = true;
        cudaGetLastError();  // clear a capture error; fall back to direct launches
    }
}

// One lagged step: traced, graph or direct launches (all issue the same kernels on the same data).
cudaError_t launch_step(rafem_ctx* c) {
    if (c->tracing) return enqueue_step_traced(c);
    ensure_graph(c);
    if (c->graph) return cudaGraphLaunch(c->graph, c->stream);
    return enqueue_step(c);
}

// ---- checkpoints of the differentiation tape: T, V and their predictor histories (8 x N doubles), StatsDev,
// istats
size_t state_bytes(const rafem_ctx* c) {
    const size_t fields = 8 + (c->proj_D ? proj_stride(c->proj_k) : 0);
    return fields * (size_t)c->N * sizeof(double) + sizeof(StatsDev) + (size_t)c->n_inst * sizeof(rafem_step_stats);
}

cudaError_t state_copy(rafem_ctx* c, void* buf, bool save) {
    char* p = static_cast<char*>(buf);
    const size_t nb = (size_t)c->N * sizeof(double);
    double* f[8] = {c->T, c->V, c->T_hist, c->V_hist, c->T_hist2, c->V_hist2, c->T_hist3, c->V_hist3};
    cudaError_t e;
    for (int q = 0; q < 8; ++q) {
        e = save ? cudaMemcpyAsync(p + q * nb, f[q], nb, cudaMemcpyDeviceToDevice, c->stream)
                 : cudaMemcpyAsync(f[q], p + q * nb, nb, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
    }
    p += 8 * nb;
    if (c->proj_D) {  // the projection predictor's history: the previous call's basis
        const size_t rb = (size_t)proj_stride(c->proj_k) * nb;
        e = save ? cudaMemcpyAsync(p, c->proj_D, rb, cudaMemcpyDeviceToDevice, c->stream)
                 : cudaMemcpyAsync(c->proj_D, p, rb, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
        p += rb;
    }
    e = save ? cudaMemcpyAsync(p, c->stats, sizeof(StatsDev), cudaMemcpyDeviceToDevice, c->stream)
             : cudaMemcpyAsync(c->stats, p, sizeof(StatsDev), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
    p += sizeof(StatsDev);
    const size_t ib = (size_t)c->n_inst * sizeof(rafem_step_stats);
    return save ? cudaMemcpyAsync(p, c->istats, ib, cudaMemcpyDeviceToDevice, c->stream)
                : cudaMemcpyAsync(c->istats, p, ib, cudaMemcpyDeviceToDevice, c->stream);
}

int tape_save(rafem_ctx* c, size_t k) {
    while (c->ckpt.size() <= k) {
        char* q = nullptr;
        CK(dalloc(c, &q, state_bytes(c)));
        c->ckpt.push_back(q);
    }
    CK(state_copy(c, c->ckpt[k], true));
    c->n_ckpt = k + 1;
    return RAFEM_OK;
}

// After a step that brought the context to step `now`: store a checkpoint when the tape asks for one.
int tape_record(rafem_ctx* c, int64_t now) {
    if (c->tape_every <= 0) return RAFEM_OK;
    const int64_t rel = now - c->tape_origin;
    if (rel <= 0 || rel % c->tape_every) return RAFEM_OK;
    return tape_save(c, (size_t)(rel / c->tape_every));
}

int finish(rafem_ctx* c, rafem_step_stats* out, bool worst) {
    StatsDev h;
    CK(cudaMemcpyAsync(&h, c->stats, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (worst) h.cur.status = h.worst;
    c->step = h.cur.step;
    if (out) *out = h.cur;
    return h.cur.status;
}

}  // namespace

extern "C" {

void rafem_default_params(rafem_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->alpha_sigma = 0.015;
    p->rho_c = 3.6e6;
    p->perf = 2.4e4;
    p->T_a = 37.0;
    p->dt = 1.0;
    p->tol = 1e-10;
    p->inner_tol = 1e-4;
    p->corrector_tol = 1e-6;
    p->max_iter = 20000;
    p->max_refine = 30;
    p->n_corrector = 1;
    p->precond = RAFEM_PRECOND_JACOBI;
    p->precision = RAFEM_PRECISION_FP64;
    p->solver = RAFEM_SOLVER_PCG;
    p->lanes_per_row = 0;
    p->rows_per_tile = 0;
    p->assembly = RAFEM_ASSEMBLY_GATHER;
    p->predictor = RAFEM_PREDICT_PROJECT;
}

const char* rafem_status_string(int s) {
    switch (s) {
        case RAFEM_OK: return "OK";
        case RAFEM_NOT_CONVERGED: return "NOT_CONVERGED";
        case RAFEM_ERR_BAD_INPUT: return "ERR_BAD_INPUT";
        case RAFEM_ERR_BAD_MESH: return "ERR_BAD_MESH";
        case RAFEM_ERR_OOM: return "ERR_OOM";
        case RAFEM_ERR_NONFINITE: return "ERR_NONFINITE";
        case RAFEM_ERR_TIMEOUT: return "ERR_TIMEOUT";
        case RAFEM_ERR_CUDA: return "ERR_CUDA";
        case RAFEM_ERR_INTERNAL: return "ERR_INTERNAL";
        case RAFEM_ERR_BREAKDOWN: return "ERR_BREAKDOWN";
        default: return "UNKNOWN";
    }
}

void rafem_destroy(rafem_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->corr_graph) cudaGraphExecDestroy(c->corr_graph);
    if (c->io_graph) cudaGraphExecDestroy(c->io_graph);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->io_ev)
        if (e) cudaEventDestroy(e);
    if (c->io_stream) cudaStreamDestroy(c->io_stream);
    for (void* p : c->tile_allocs) cudaFree(p);
    for (void* p : c->allocs) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// Work tiles of the persistent solvers: contiguous row ranges of at most rows_per_tile rows (a multiple of 32
// for SELL-32), never straddling instances. rows_per_tile <= 0 picks one tile per block for a single instance
// and about four per block for a batch. Replaces any previous tiles and drops the captured step graph.
static int build_tiles(rafem_ctx* c, int rows_per_tile) {
    const int N = c->N, n_inst = c->n_inst;
    const std::vector<int32_t>& node_off = c->inst_node_off;
    if (rows_per_tile <= 0)
        rows_per_tile = n_inst == 1 ? (N + c->maxb - 1) / c->maxb : (N + 4 * c->maxb - 1) / (4 * c->maxb);
    rows_per_tile = std::max(rows_per_tile, 1);
    if (c->sell) rows_per_tile = (rows_per_tile + SELL_C - 1) / SELL_C * SELL_C;
    std::vector<int32_t> t0, t1, ti, it0(n_inst), it1(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        it0[i] = (int32_t)t0.size();
        for (int64_t r = node_off[i]; r < node_off[i + 1]; r += rows_per_tile) {
            t0.push_back((int32_t)r);
            t1.push_back((int32_t)std::min<int64_t>(r + rows_per_tile, node_off[i + 1]));
            ti.push_back(i);
        }
        it1[i] = (int32_t)t0.size();
    }
    cudaStream_t st = c->stream;
    CK(cudaStreamSynchronize(st));
    drop_graphs(c);  // the captured graphs hold the tile arrays freed below
    for (void* p : c->tile_allocs) cudaFree(p);
    c->tile_allocs.clear();
    const int nt = (int)t0.size();
    auto talloc = [&](auto** ptr, size_t count) -> cudaError_t {
        void* q = nullptr;
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(**ptr) + 64;
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return e;
        c->tile_allocs.push_back(q);
        *ptr = static_cast<std::remove_reference_t<decltype(*ptr)>>(q);
        return cudaMemsetAsync(q, 0, bytes, st);
    };
    CK(talloc(&c->tile_r0, nt));
    CK(talloc(&c->tile_r1, nt));
    CK(talloc(&c->tile_inst, nt));
    CK(talloc(&c->inst_t0, n_inst));
    CK(talloc(&c->inst_t1, n_inst));
    CK(talloc(&c->partial, (size_t)kPartialQ * nt));
    int max_rows = 1;
    for (int t = 0; t < nt; ++t) max_rows = std::max(max_rows, t1[t] - t0[t]);
    c->proj_sub = (max_rows + kProjChunk - 1) / kProjChunk;
    CK(talloc(&c->proj_partial, (size_t)kProjQ * nt * c->proj_sub));
    CK(cudaMemcpyAsync(c->tile_r0, t0.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->tile_r1, t1.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->tile_inst, ti.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->inst_t0, it0.data(), n_inst * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->inst_t1, it1.data(), n_inst * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // host vectors go out of scope
    c->n_tiles = nt;
    c->grid = std::min(nt, c->maxb);
    c->rows_per_tile = rows_per_tile;
    return RAFEM_OK;
}

static int create_impl(const rafem_mesh* m, const rafem_params* prm, void* stream, rafem_ctx* c, int n_inst,
                       const std::vector<int32_t>& node_off) {
    const int N = m->n_nodes, E = m->n_tets;
    if ((int64_t)E * 16 >= (int64_t)INT32_MAX) return RAFEM_ERR_BAD_INPUT;  // slot codes and 4 e + a incidence
    c->n_inst = n_inst;
    c->inst_node_off = node_off;
    c->prm = *prm;
    c->N = N;
    c->E = E;
    CK(cudaGetDevice(&c->device));
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    // ---- host setup
    std::vector<int8_t> orient;
    double vol_min = 0.0, vol_max = 0.0;
    int v = validate_mesh(N, E, m->tets, m->coords, orient, &vol_min, &vol_max);
    if (v == -1) return RAFEM_ERR_BAD_INPUT;
    if (v == -2) return RAFEM_ERR_BAD_MESH;
    for (int64_t i = 0; i < 3LL * N; ++i)
        if (!std::isfinite(m->coords[i])) return RAFEM_ERR_NONFINITE;
    for (int64_t e = 0; e < E; ++e)
        if (!std::isfinite(m->sigma0[e]) || !std::isfinite(m->k[e])) return RAFEM_ERR_NONFINITE;
    for (int64_t i = 0; i < N; ++i)
        if ((m->bc_V[i] && !std::isfinite(m->g_V[i])) || (m->bc_T[i] && !std::isfinite(m->g_T[i])))
            return RAFEM_ERR_NONFINITE;
    std::vector<int32_t> rp, col;
    build_pattern(N, E, m->tets, rp, col);
    c->nnz = (int64_t)col.size();
    if (c->nnz >= (int64_t)SLOT_MASK) return RAFEM_ERR_BAD_INPUT;
    std::vector<int32_t> color;
    c->n_colors = color_elements(N, E, m->tets, color);
    if (c->n_colors <= 0) return RAFEM_ERR_INTERNAL;
    std::vector<int64_t> order(E);
    {
        std::vector<int64_t> cnt(c->n_colors + 1, 0);
        for (int64_t e = 0; e < E; ++e) cnt[color[e] + 1]++;
        for (int q = 0; q < c->n_colors; ++q) cnt[q + 1] += cnt[q];
        c->color_off.assign(cnt.begin(), cnt.end());
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t e = 0; e < E; ++e) order[pos[color[e]]++] = e;
    }
    std::vector<int32_t> slots;
    build_slots(E, m->tets, rp, col, order, slots);
    std::vector<int32_t> diag(N);
    for (int i = 0; i < N; ++i) {
        const int32_t* f = std::lower_bound(col.data() + rp[i], col.data() + rp[i + 1], i);
        diag[i] = (int32_t)(f - col.data());
    }
    // storage layout of the matrix values: SELL-32 (lanes_per_row 0 or 1) or CSR
    c->lanes = prm->lanes_per_row ? prm->lanes_per_row : 1;
    c->sell = c->lanes == 1;
    const bool want16 = prm->lanes_per_row == 0;
    c->gather = c->sell && prm->assembly == RAFEM_ASSEMBLY_GATHER;
    {
        // double-word passes: the element constants and fields must sit well inside the float exponent range so
        // that the low words keep their 24 bits (volumes, and through them the G entries, drive the smallest ones)
        const double big = std::ldexp(1.0, 60);
        double amax = std::max({std::fabs(prm->alpha_sigma), std::fabs(prm->T_a), prm->perf, prm->rho_c / prm->dt});
        for (int64_t e = 0; e < E; ++e) amax = std::max(amax, std::fabs(m->sigma0[e]));
        for (int64_t i = 0; i < N; ++i) amax = std::max({amax, std::fabs(m->g_V[i]), std::fabs(m->g_T[i])});
        const bool scales_ok = vol_min >= std::ldexp(1.0, -90) && vol_max <= big && amax <= big &&
                               prm->rho_c / prm->dt >= std::ldexp(1.0, -30);
        if (prm->arith == RAFEM_ARITH_DW && (!c->gather || !scales_ok)) return RAFEM_ERR_BAD_INPUT;
        c->dw = c->gather && scales_ok && prm->arith != RAFEM_ARITH_FP64;
    }
    // element storage order. The colour scatter needs the elements of a colour stored contiguously; the row-owner
    // assembly does not, so there the elements are stored by their smallest node (a counting sort, stable in mesh
    // order), which keeps the nodal gathers of the element passes local. The colour pass over the thermal matrix
    // then walks a list of storage indices (clist) in colour order, and the slot codes keep the first/last-writer
    // flags of that colour order.
    std::vector<int32_t> clist;
    if (c->gather) {
        std::vector<int64_t> cnt(N + 1, 0), store(E);
        std::vector<int32_t> key(E);
        for (int64_t e = 0; e < E; ++e) {
            const int32_t* t = m->tets + 4 * e;
            key[e] = std::min(std::min(t[0], t[1]), std::min(t[2], t[3]));
            cnt[key[e] + 1]++;
        }
        for (int i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
        std::vector<int32_t> pos_store(E);
        for (int64_t e = 0; e < E; ++e) {
            const int64_t q = cnt[key[e]]++;
            store[q] = e;
            pos_store[e] = (int32_t)q;
        }
        std::vector<int32_t> slots_store(slots.size());
        clist.resize(E);
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < E; ++p) {
            const int32_t q = pos_store[order[p]];
            clist[p] = q;
            for (int k = 0; k < 16; ++k) slots_store[(size_t)k * E + q] = slots[(size_t)k * E + p];
        }
        slots.swap(slots_store);
        order.swap(store);
    }
    std::vector<int32_t> dev_rp, dev_ci;
    std::vector<int16_t> d16;
    std::vector<int32_t> g_off, g_cnt, g_elem, i_off, i_cnt, i_elem;
    std::vector<uint8_t> g_idx, g_cab;
    std::vector<int32_t> pat_off, pat_pool;
    bool patterns = false;
    if (c->sell) {
        std::vector<int32_t> map;
        // one column pattern per slice where that widens no slice (lattice-like numberings), else per-entry columns
        patterns = build_sell_patterns(N, rp, col, dev_rp, dev_ci, map, pat_off, pat_pool);
        if (!patterns) build_sell(N, rp, col, dev_rp, dev_ci, map);
        if (c->gather)
            build_gather(N, E, rp, col, slots, dev_rp, map, g_off, g_cnt, g_elem, g_idx,
                         prm->coupling == RAFEM_COUPLING_MONOLITHIC ? &g_cab : nullptr);
        if (want16) {
            bool fits = true;
            d16.resize(dev_ci.size());
            const int S = (int)dev_rp.size() - 1;
            for (int sl = 0; sl < S && fits; ++sl)
                for (int32_t q = dev_rp[sl]; q < dev_rp[sl + 1]; ++q) {
                    const int r = sl * SELL_C + (int)((q - dev_rp[sl]) % SELL_C);
                    const int d = dev_ci[q] - r;
                    if (d < -32768 || d > 32767) {
                        fits = false;
                        break;
                    }
                    d16[q] = (int16_t)d;
                }
            if (fits) c->lanes = 2;
            else d16.clear();
        }
        if (patterns) c->lanes = 3;
        c->nnz_store = (int64_t)dev_ci.size();
        if (c->nnz_store >= (int64_t)SLOT_MASK) return RAFEM_ERR_BAD_INPUT;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < (int64_t)slots.size(); ++q) {
            const int32_t code = slots[q];
            slots[q] = map[code & SLOT_MASK] | (code & ~SLOT_MASK);
        }
        for (int i = 0; i < N; ++i) diag[i] = map[diag[i]];
        c->h_map = std::move(map);
    } else {
        dev_rp = rp;
        dev_ci = col;
        c->nnz_store = c->nnz;
    }
    IluHost ih;
    if (prm->precond == RAFEM_PRECOND_ILU0) {
        if (n_inst != 1) return RAFEM_ERR_BAD_INPUT;
        if (build_ilu(N, rp, col, prm->ilu_order, ih) != 0) return RAFEM_ERR_BAD_INPUT;
        c->ilu = true;
        c->ilu_pmap_csr = ih.pmap;
        c->ilu_perm = ih.perm;
        if (c->sell)
            for (auto& q : ih.pmap)
                if (q >= 0) q = c->h_map[q];
    }
    std::vector<int32_t> nodes_soa(4LL * E);
    std::vector<double> sig_s(E), k_s(E);
    for (int64_t ep = 0; ep < E; ++ep) {
        const int64_t e = order[ep];
        for (int a = 0; a < 4; ++a) nodes_soa[(size_t)a * E + ep] = m->tets[4 * e + a];
        sig_s[ep] = m->sigma0[e];
        k_s[ep] = m->k[e];
    }
    if (c->gather) build_incidence(N, E, nodes_soa, i_off, i_cnt, i_elem);
    std::vector<int32_t> order32(order.begin(), order.end());
    // ---- device buffers
    const size_t nnz = (size_t)c->nnz_store;
    // FP32 copies of the matrices and the FP32 Krylov vectors: the mixed-precision solves, and the monolithic
    // step's flexible GMRES, whose preconditioner solves run in mixed precision
    const bool mixed = prm->precision == RAFEM_PRECISION_MIXED ||
                       (prm->coupling == RAFEM_COUPLING_MONOLITHIC && prm->coupled_solver == RAFEM_COUPLED_FGMRES);
    CK(dalloc(c, &c->rp, dev_rp.size()));
    CK(dalloc(c, &c->ci, nnz));
    CK(dalloc(c, &c->diag, N));
    CK(dalloc(c, &c->e_nodes, 4 * (size_t)E));
    CK(dalloc(c, &c->e_slots, 16 * (size_t)E));
    CK(dalloc(c, &c->e_G, 10 * (size_t)E));
    CK(dalloc(c, &c->e_vol, E));
    CK(dalloc(c, &c->e_sig0, E));
    CK(dalloc(c, &c->e_k, E));
    CK(dalloc(c, &c->xyz, 3 * (size_t)N));
    CK(dalloc(c, &c->bcV, N));
    CK(dalloc(c, &c->bcT, N));
    CK(dalloc(c, &c->gV, N));
    CK(dalloc(c, &c->gT, N));
    CK(dalloc(c, &c->valsV, nnz));
    CK(dalloc(c, &c->valsT, nnz));
    if (mixed) {
        CK(dalloc(c, &c->valsV32, nnz));
        CK(dalloc(c, &c->valsT32, nnz));
    }
    CK(dalloc(c, &c->bV, N));
    CK(dalloc(c, &c->bT, N));
    CK(dalloc(c, &c->bTc, N));
    CK(dalloc(c, &c->V, N));
    CK(dalloc(c, &c->T, N));
    CK(dalloc(c, &c->T_old, N));
    CK(dalloc(c, &c->T_prev, N));
    CK(dalloc(c, &c->V_hist, N));
    CK(dalloc(c, &c->T_hist, N));
    CK(dalloc(c, &c->V_hist2, N));
    CK(dalloc(c, &c->T_hist2, N));
    CK(dalloc(c, &c->V_hist3, N));
    CK(dalloc(c, &c->T_hist3, N));
    CK(dalloc(c, &c->wr, N));
    CK(dalloc(c, &c->wu, N));
    CK(dalloc(c, &c->ww, N));
    CK(dalloc(c, &c->wp, N));
    CK(dalloc(c, &c->ws, N));
    CK(dalloc(c, &c->wdinv, N));
    if (mixed) {
        CK(dalloc(c, &c->fr, N));
        CK(dalloc(c, &c->fu, N));
        CK(dalloc(c, &c->fw, N));
        CK(dalloc(c, &c->fp, N));
        CK(dalloc(c, &c->fs, N));
        CK(dalloc(c, &c->fd, N));
        CK(dalloc(c, &c->fdinv, N));
    }
    if (prm->solver == RAFEM_SOLVER_PIPECG)
        for (double** v : {&c->pz, &c->pq, &c->pm0, &c->pm1}) CK(dalloc(c, v, N));
    CK(dalloc(c, &c->stats, 1));
    CK(dalloc(c, &c->scratch, 8));
    CK(dalloc(c, &c->instV, n_inst));
    CK(dalloc(c, &c->instT, n_inst));
    CK(dalloc(c, &c->istats, n_inst));
    CK(dalloc(c, &c->bar, 1));
    CK(dalloc(c, &c->e_order, E));
    CK(dalloc(c, &c->corr, 1));
    CK(dalloc(c, &c->proj_coef, (size_t)kProjMax * n_inst));
    CK(dalloc(c, &c->proj_kin, n_inst));
    CK(dalloc(c, &c->proj_kout, n_inst));
    if (prm->predictor == RAFEM_PREDICT_PROJECT) {
        c->proj_k = prm->proj_basis > 0 ? prm->proj_basis : kProjDefault;
        const size_t nd = (size_t)proj_stride(c->proj_k) * N;
        CK(dalloc(c, &c->proj_D, nd + 8));
        CK(dalloc(c, &c->proj_Y, nd + 8));
        CK(dalloc(c, &c->proj_r0, N));
        CK(cudaMemsetAsync(c->proj_D, 0, nd * sizeof(double), c->stream));
    }
    CK(dalloc(c, &c->V_old, N));
    CK(dalloc(c, &c->stats_save, 1));
    CK(dalloc(c, &c->istats_save, n_inst));
    if (!clist.empty()) {
        CK(dalloc(c, &c->e_clist, E));
        CK(cudaMemcpyAsync(c->e_clist, clist.data(), E * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    }
    // ---- uploads
    cudaStream_t st = c->stream;
    CK(cudaMemcpyAsync(c->rp, dev_rp.data(), dev_rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->ci, dev_ci.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    if (!d16.empty()) {
        CK(dalloc(c, &c->ci16, d16.size()));
        CK(cudaMemcpyAsync(c->ci16, d16.data(), d16.size() * sizeof(int16_t), cudaMemcpyHostToDevice, st));
    }
    if (patterns) {
        CK(dalloc(c, &c->pat_off, pat_off.size()));
        CK(dalloc(c, &c->pat_pool, pat_pool.size()));
        CK(cudaMemcpyAsync(c->pat_off, pat_off.data(), pat_off.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(c->pat_pool, pat_pool.data(), pat_pool.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                           st));
    }
    CK(cudaMemcpyAsync(c->diag, diag.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->e_nodes, nodes_soa.data(), nodes_soa.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->e_slots, slots.data(), slots.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->e_order, order32.data(), E * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->e_sig0, sig_s.data(), E * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->e_k, k_s.data(), E * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->xyz, m->coords, 3 * (size_t)N * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->bcV, m->bc_V, N, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->bcT, m->bc_T, N, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->gV, m->g_V, N * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->gT, m->g_T, N * sizeof(double), cudaMemcpyHostToDevice, st));
    if (c->gather) {
        int32_t *goff, *gcnt, *celem, *ioff, *icnt, *ielem;
        uint8_t* cg;
        double *cval, *ework, *mT;
        CK(dalloc(c, &goff, g_off.size()));
        CK(dalloc(c, &gcnt, g_cnt.size()));
        CK(dalloc(c, &celem, g_elem.size()));
        CK(dalloc(c, &cg, g_idx.size()));
        if (c->dw) {
            cval = nullptr;
            CK(dalloc(c, &c->gdw.cval, g_elem.size()));
            CK(dalloc(c, &c->gdw.tq, 7 * (size_t)E));
            CK(dalloc(c, &c->gdw.Ts, N));
            CK(dalloc(c, &c->gdw.To, N));
            CK(dalloc(c, &c->gdw.V, N));
        } else {
            CK(dalloc(c, &cval, g_elem.size()));
        }
        CK(dalloc(c, &ioff, i_off.size()));
        CK(dalloc(c, &icnt, i_cnt.size()));
        CK(dalloc(c, &ielem, i_elem.size()));
        CK(dalloc(c, &ework, E));
        CK(dalloc(c, &mT, N));
        CK(cudaMemcpyAsync(goff, g_off.data(), g_off.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(gcnt, g_cnt.data(), g_cnt.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(celem, g_elem.data(), g_elem.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(cg, g_idx.data(), g_idx.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ioff, i_off.data(), i_off.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(icnt, i_cnt.data(), i_cnt.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(ielem, i_elem.data(), i_elem.size() * 4, cudaMemcpyHostToDevice, st));
        c->gd.goff = goff;
        c->gd.gcnt = gcnt;
        c->gd.cval = cval;
        c->gd.celem = celem;
        c->gd.ioff = ioff;
        c->gd.icnt = icnt;
        c->gd.ielem = ielem;
        c->gd.ework = ework;
        c->gd.mT = mT;
        c->gather_cg = cg;
        c->gather_nc = (long long)g_elem.size();
        if (!g_cab.empty()) {
            CK(dalloc(c, &c->mg.cab, g_cab.size()));
            CK(dalloc(c, &c->mg.Gc, g_cab.size()));
            CK(dalloc(c, &c->mg.tc, (size_t)dev_rp.back()));
            CK(dalloc(c, &c->mg.rec, 4 * (size_t)E));
            CK(dalloc(c, &c->mg.rt, 4 * (size_t)E));
            CK(cudaMemcpyAsync(c->mg.cab, g_cab.data(), g_cab.size(), cudaMemcpyHostToDevice, st));
        }
    }
    c->el.E = E;
    c->el.nodes = c->e_nodes;
    c->el.slots = c->e_slots;
    c->el.G = c->e_G;
    c->el.vol = c->e_vol;
    c->el.sigma0 = c->e_sig0;
    c->el.k = c->e_k;
    // ---- solver schedule: one tile per co-resident block (SELL tiles start on a slice boundary)
    int block = 0;
    int maxb = krylov_max_blocks(c->lanes, prm->precision, prm->solver == RAFEM_SOLVER_PIPECG, &block);
    if (maxb <= 0) return RAFEM_ERR_BAD_INPUT;
    if (prm->coupling == RAFEM_COUPLING_MONOLITHIC && prm->coupled_solver == RAFEM_COUPLED_FGMRES) {
        // the preconditioner's inner solves launch the mixed-precision kernel as well: prepare it (its dynamic
        // shared memory) and keep the schedule within what both kernels hold co-resident
        const int mb2 = krylov_max_blocks(c->lanes, RAFEM_PRECISION_MIXED, false, nullptr);
        if (mb2 <= 0) return RAFEM_ERR_BAD_INPUT;
        maxb = std::min(maxb, mb2);
    }
    c->block = block;
    c->maxb = maxb;
    {
        const int t = build_tiles(c, prm->rows_per_tile);
        if (t != RAFEM_OK) return t;
    }
    if (prm->solver == RAFEM_SOLVER_GMRES) {
        if (n_inst != 1 || !c->sell) return RAFEM_ERR_BAD_INPUT;
        c->gm_m = prm->gmres_restart > 0 ? prm->gmres_restart : 30;
        c->gm_ld = (N + SELL_C - 1) / SELL_C * SELL_C;
        CK(dalloc(c, &c->gm_V, (size_t)c->gm_m * c->gm_ld + SELL_C));
        for (double** v : {&c->gm_w0, &c->gm_w1, &c->gm_z, &c->gm_dinv}) CK(dalloc(c, v, (size_t)N + SELL_C));
        c->gm_grid = gmres_max_blocks(c->gm_m);
        if (c->gm_grid <= 0) return RAFEM_ERR_CUDA;
        c->gm_grid = std::min(c->gm_grid, (N + SELL_C - 1) / SELL_C);
        CK(dalloc(c, &c->gm_partial, (size_t)gmres_partial_slots(c->gm_m) * c->gm_grid));
        CK(dalloc(c, &c->gm_H, (size_t)c->gm_grid * (c->gm_m + 1) * c->gm_m));
    }
    if (prm->coupling == RAFEM_COUPLING_MONOLITHIC) {
        if (n_inst != 1 || !c->sell) return RAFEM_ERR_BAD_INPUT;
        c->mono = true;
        const size_t n2 = 2 * (size_t)N + 2 * SELL_C;
        CK(dalloc(c, &c->m_vals4, 4 * (size_t)c->nnz_store));
        for (double** v : {&c->m_R, &c->m_D, &c->mb_r, &c->mb_rh, &c->mb_p, &c->mb_ph, &c->mb_v, &c->mb_s, &c->mb_sh,
                           &c->mb_t})
            CK(dalloc(c, v, n2));
        CK(dalloc(c, &c->mb_dinv, 2 * n2));
        c->mb_grid = bicgstab_max_blocks(2);
        if (c->mb_grid <= 0) return RAFEM_ERR_CUDA;
        CK(dalloc(c, &c->mb_partial, (size_t)bicgstab_partial_slots() * c->mb_grid));
        if (prm->coupled_solver == RAFEM_COUPLED_FGMRES) {
            c->fg_ld = (2 * (size_t)N + 63) / 64 * 64;
            c->fg_G = fg_grid();
            if (c->fg_G <= 0) return RAFEM_ERR_CUDA;
            CK(dalloc(c, &c->fg_V, (size_t)(kFgMax + 1) * c->fg_ld));
            CK(dalloc(c, &c->fg_Z, (size_t)kFgMax * c->fg_ld));
            CK(dalloc(c, &c->fg_w, c->fg_ld));
            for (double** v : {&c->fg_rV, &c->fg_rT, &c->fg_zV, &c->fg_zT}) CK(dalloc(c, v, (size_t)N + SELL_C));
            CK(dalloc(c, &c->fg_partial, (size_t)(kFgMax + 2) * c->fg_G));
            void* stp = nullptr;
            CK(cudaMalloc(&stp, sizeof(FgState)));
            c->allocs.push_back(stp);
            c->fg_st = static_cast<FgState*>(stp);
            const int32_t one = 1;
            CK(dalloc(c, &c->fg_one, 1));
            CK(cudaMemcpyAsync(c->fg_one, &one, sizeof(one), cudaMemcpyHostToDevice, st));
        }
    }
    if (prm->solver == RAFEM_SOLVER_BICGSTAB) {
        if (n_inst != 1 || !c->sell) return RAFEM_ERR_BAD_INPUT;
        for (double** v : {&c->bg_r, &c->bg_rh, &c->bg_p, &c->bg_ph, &c->bg_v, &c->bg_s, &c->bg_sh, &c->bg_t,
                           &c->bg_dinv})
            CK(dalloc(c, v, (size_t)N + SELL_C));
        c->bg_grid = bicgstab_max_blocks(1);
        if (c->bg_grid <= 0) return RAFEM_ERR_CUDA;
        CK(dalloc(c, &c->bg_partial, (size_t)bicgstab_partial_slots() * c->bg_grid));
    }
    if (c->ilu) {
        const size_t nz = ih.sc.size(), Np = (size_t)ih.Np;
        int32_t *lvl, *sp, *sc, *pm, *pr;
        uint8_t *rl, *dk;
        CK(dalloc(c, &lvl, ih.lvl.size()));
        CK(dalloc(c, &sp, ih.sp.size()));
        CK(dalloc(c, &sc, nz));
        CK(dalloc(c, &pm, nz));
        CK(dalloc(c, &pr, Np));
        CK(dalloc(c, &rl, Np));
        CK(dalloc(c, &dk, Np));
        CK(cudaMemcpyAsync(lvl, ih.lvl.data(), ih.lvl.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(sp, ih.sp.data(), ih.sp.size() * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(sc, ih.sc.data(), nz * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(pm, ih.pmap.data(), nz * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(pr, ih.perm.data(), Np * 4, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(rl, ih.rlen.data(), Np, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dk, ih.dk.data(), Np, cudaMemcpyHostToDevice, st));
        c->il.Np = ih.Np;
        c->il.n_levels = ih.n_levels;
        c->il.nnz = (long long)nz;
        c->il.lvl = lvl;
        c->il.sp = sp;
        c->il.sc = sc;
        c->il.pmap = pm;
        c->il.rlen = rl;
        c->il.dk = dk;
        c->il.perm = pr;
        c->il.h_lvl = ih.lvl;
        CK(dalloc(c, &c->ilu_AV, nz));
        CK(dalloc(c, &c->ilu_FV, nz));
        CK(dalloc(c, &c->ilu_AT, nz));
        CK(dalloc(c, &c->ilu_FT, nz));
        CK(dalloc(c, &c->ilu_DV, Np));
        CK(dalloc(c, &c->ilu_DT, Np));
        // the ring solver's layouts of P A P^T, L and U (values split from the combined layout per refactorisation)
        IluRingHost irh;
        build_ilu_ring(ih, irh);
        IluRingDev d;
        d.Np = ih.Np;
        d.n_levels = ih.n_levels;
        d.patterns = irh.A.patterns && irh.L.patterns && irh.U.patterns;
        d.lvl = lvl;
        d.perm = pr;
        auto upload = [&](const std::vector<int32_t>& v, const int32_t** dst) -> cudaError_t {
            int32_t* q = nullptr;
            cudaError_t e = dalloc(c, &q, v.size());
            if (e == cudaSuccess && !v.empty())
                e = cudaMemcpyAsync(q, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
            *dst = q;
            return e;
        };
        for (auto pr2 : {std::make_pair(&irh.A, &d.A), std::make_pair(&irh.L, &d.L), std::make_pair(&irh.U, &d.U)}) {
            CK(upload(pr2.first->sp, &pr2.second->sp));
            CK(upload(pr2.first->sc, &pr2.second->sc));
            CK(upload(pr2.first->src, &pr2.second->src));
            if (d.patterns) {
                CK(upload(pr2.first->pat_off, &pr2.second->pat_off));
                CK(upload(pr2.first->pat_pool, &pr2.second->pat_pool));
            }
        }
        d.nA = (long long)irh.A.sc.size();
        d.nL = (long long)irh.L.sc.size();
        d.nU = (long long)irh.U.sc.size();
        const bool mixed = prm->precision == RAFEM_PRECISION_MIXED;
        for (double** v : {&d.xv, &d.bv, &d.r64, &d.z64, &d.p64, &d.q64}) CK(dalloc(c, v, Np));
        if (mixed)
            for (float** v : {&d.r32, &d.z32, &d.p32, &d.q32, &d.d32}) CK(dalloc(c, v, Np));
        c->ir_grid = ilu_ring_max_blocks();
        if (c->ir_grid <= 0) return RAFEM_ERR_CUDA;
        CK(dalloc(c, &d.partial, (size_t)kIluRingSlots * c->ir_grid));
        for (int sys = 0; sys < 2; ++sys) {
            c->ir[sys] = d;
            IluRingDev& e = c->ir[sys];
            CK(dalloc(c, &e.A64, (size_t)d.nA));
            if (mixed) {
                CK(dalloc(c, &e.A32, (size_t)d.nA));
                CK(dalloc(c, &e.L32, (size_t)d.nL));
                CK(dalloc(c, &e.U32, (size_t)d.nU));
                CK(dalloc(c, &e.dinv32, Np));
            } else {
                CK(dalloc(c, &e.L64, (size_t)d.nL));
                CK(dalloc(c, &e.U64, (size_t)d.nU));
            }
        }
        CK(cudaStreamSynchronize(st));  // host layouts go out of scope
    }
    // ---- device-side setup: geometry, constant thermal system, Dirichlet identity rows, initial fields
    CK(launch_geometry(c->el, c->xyz, c->e_G, c->e_vol, st));
    if (c->dw) {
        CK(launch_fill_dw(c->gdw, c->gather_nc, c->gd.celem, c->gather_cg, c->el, prm->rho_c / prm->dt, st));
        CK(launch_node_mass(c->gd, N, c->e_vol, prm->rho_c / prm->dt, st));
    } else if (c->gather) {
        CK(launch_fill_cval(c->gather_nc, c->gd.celem, c->gather_cg, c->e_sig0, c->e_G, E, const_cast<double*>(c->gd.cval),
                            st));
        CK(launch_node_mass(c->gd, N, c->e_vol, prm->rho_c / prm->dt, st));
    }
    if (c->mg.cab)
        CK(launch_coupled_fill(c->mg, c->gd, c->gather_nc, N, c->rp, c->diag, c->el, prm->rho_c / prm->dt + prm->perf,
                               true, st));
    CK(launch_set_dirichlet_identity(N, c->bcV, c->diag, c->valsV, c->valsV32, st));
    CK(launch_set_dirichlet_identity(N, c->bcT, c->diag, c->valsT, c->valsT32, st));
    const double c_matrix = prm->rho_c / prm->dt + prm->perf;
    for (int q = 0; q < c->n_colors; ++q)
        CK(launch_assemble_T(c->el, c->color_off[q], c->color_off[q + 1], c->bcT, c->gT, c_matrix,
                             prm->perf * prm->T_a, c->valsT, c->valsT32, c->bTc, prm->lift, c->e_clist, st));
    if (c->ilu) CK(ilu_refactor(c, RAFEM_SYS_T, st));
    k_init_fields<<<(N + 255) / 256, 256, 0, st>>>(N, prm->T_a, c->bcT, c->gT, c->bcV, c->gV, c->T, c->V);
    CK(cudaGetLastError());
    k_set_step<<<1, 1, 0, st>>>(c->stats, 0);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    c->h_rp = std::move(rp);
    c->h_col = std::move(col);
    return RAFEM_OK;
}

static int validate_params(const rafem_mesh* m, const rafem_params* prm) {
    if (!m || !prm || !m->coords || !m->tets || !m->bc_V || !m->g_V || !m->bc_T || !m->g_T || !m->sigma0 || !m->k)
        return RAFEM_ERR_BAD_INPUT;
    if (m->n_nodes < 4 || m->n_tets < 1) return RAFEM_ERR_BAD_INPUT;
    if (!(prm->dt > 0) || !(prm->rho_c > 0) || !(prm->perf >= 0) || !(prm->tol > 0) || prm->max_iter < 1 ||
        prm->n_corrector < 1 || prm->n_corrector > 50)
        return RAFEM_ERR_BAD_INPUT;
    if (prm->lanes_per_row != 0 && prm->lanes_per_row != 1 && prm->lanes_per_row != 4 && prm->lanes_per_row != 8 &&
        prm->lanes_per_row != 16 && prm->lanes_per_row != 32)
        return RAFEM_ERR_BAD_INPUT;
    if (prm->precision != RAFEM_PRECISION_FP64 && prm->precision != RAFEM_PRECISION_MIXED) return RAFEM_ERR_BAD_INPUT;
    if (prm->precision == RAFEM_PRECISION_MIXED && !(prm->inner_tol > 0 && prm->inner_tol < 1)) return RAFEM_ERR_BAD_INPUT;
    if (prm->precond != RAFEM_PRECOND_JACOBI && prm->precond != RAFEM_PRECOND_ILU0) return RAFEM_ERR_BAD_INPUT;
    if (prm->precond == RAFEM_PRECOND_ILU0 &&
        (prm->ilu_order != RAFEM_ILU_MULTICOLOR && prm->ilu_order != RAFEM_ILU_NATURAL))
        return RAFEM_ERR_BAD_INPUT;
    if (prm->solver != RAFEM_SOLVER_PCG && prm->solver != RAFEM_SOLVER_BICGSTAB && prm->solver != RAFEM_SOLVER_GMRES &&
        prm->solver != RAFEM_SOLVER_PIPECG)
        return RAFEM_ERR_BAD_INPUT;
    if (prm->solver == RAFEM_SOLVER_PIPECG &&
        (prm->precision != RAFEM_PRECISION_FP64 || prm->precond != RAFEM_PRECOND_JACOBI ||
         prm->coupling != RAFEM_COUPLING_STAGGERED))
        return RAFEM_ERR_BAD_INPUT;
    if (prm->gmres_restart < 0 || prm->gmres_restart > 64) return RAFEM_ERR_BAD_INPUT;
    if (prm->gmres_min_restart < 0 ||
        prm->gmres_min_restart > (prm->gmres_restart > 0 ? prm->gmres_restart : 30))
        return RAFEM_ERR_BAD_INPUT;
    if ((prm->solver == RAFEM_SOLVER_BICGSTAB || prm->solver == RAFEM_SOLVER_GMRES) &&
        (prm->precision != RAFEM_PRECISION_FP64 || prm->precond != RAFEM_PRECOND_JACOBI ||
         (prm->lanes_per_row != 0 && prm->lanes_per_row != 1)))
        return RAFEM_ERR_BAD_INPUT;
    if (prm->lift != RAFEM_LIFT_SYMMETRIC && prm->lift != RAFEM_LIFT_ROW) return RAFEM_ERR_BAD_INPUT;
    if (prm->predictor < 0 || prm->predictor > RAFEM_PREDICT_PROJECT) return RAFEM_ERR_BAD_INPUT;
    if (prm->proj_basis < 0 || prm->proj_basis > kProjMax) return RAFEM_ERR_BAD_INPUT;
    if (prm->coupling != RAFEM_COUPLING_STAGGERED && prm->coupling != RAFEM_COUPLING_MONOLITHIC)
        return RAFEM_ERR_BAD_INPUT;
    if (prm->coupling == RAFEM_COUPLING_MONOLITHIC &&
        (prm->precision != RAFEM_PRECISION_FP64 || (prm->lanes_per_row != 0 && prm->lanes_per_row != 1)))
        return RAFEM_ERR_BAD_INPUT;
    if (prm->coupled_solver != RAFEM_COUPLED_FGMRES && prm->coupled_solver != RAFEM_COUPLED_BICGSTAB)
        return RAFEM_ERR_BAD_INPUT;
    if (prm->lift == RAFEM_LIFT_ROW && (prm->solver == RAFEM_SOLVER_PCG || prm->solver == RAFEM_SOLVER_PIPECG))
        return RAFEM_ERR_BAD_INPUT;
    if (prm->assembly != RAFEM_ASSEMBLY_GATHER && prm->assembly != RAFEM_ASSEMBLY_COLOR) return RAFEM_ERR_BAD_INPUT;
    if (prm->arith != RAFEM_ARITH_AUTO && prm->arith != RAFEM_ARITH_FP64 && prm->arith != RAFEM_ARITH_DW)
        return RAFEM_ERR_BAD_INPUT;
    return RAFEM_OK;
}

int rafem_create(const rafem_mesh* m, const rafem_params* prm, void* stream, rafem_ctx** out) {
    if (!out) return RAFEM_ERR_BAD_INPUT;
    *out = nullptr;
    {
        const int v = validate_params(m, prm);
        if (v != RAFEM_OK) return v;
    }
    rafem_ctx* c = new (std::nothrow) rafem_ctx();
    if (!c) return RAFEM_ERR_OOM;
    int s;
    try {
        s = create_impl(m, prm, stream, c, 1, std::vector<int32_t>{0, m->n_nodes});
    } catch (const std::bad_alloc&) {
        s = RAFEM_ERR_OOM;
    }
    if (s != RAFEM_OK) {
        rafem_destroy(c);
        return s;
    }
    *out = c;
    return RAFEM_OK;
}

int rafem_assemble(rafem_ctx* c, int which) {
    if (!c || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    CK(enqueue_assemble(c, which, c->T, c->T));
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

int rafem_solve(rafem_ctx* c, int which, rafem_step_stats* stats) {
    if (!c || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    c->tape_every = 0;
    c->r0_fresh = false;  // a standalone solve starts from its own residual
    k_begin_step<<<1, 128, 0, c->stream>>>(c->stats, c->istats, c->n_inst);
    CK(cudaGetLastError());
    CK(enqueue_solve(c, which, which == RAFEM_SYS_V ? c->bV : c->bT, which == RAFEM_SYS_V ? c->V : c->T));
    k_record<<<1, 128, 0, c->stream>>>(which == RAFEM_SYS_V ? c->instV : c->instT, c->n_inst, c->bar, which, c->stats, c->istats, 0);
    CK(cudaGetLastError());
    return finish(c, stats, false);
}

int rafem_solve_rhs(rafem_ctx* c, int which, const double* b, double* x, rafem_step_stats* stats) {
    if (!c || !b || !x || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    k_begin_step<<<1, 128, 0, c->stream>>>(c->stats, c->istats, c->n_inst);
    CK(cudaGetLastError());
    CK(enqueue_solve(c, which, b, x));
    k_record<<<1, 128, 0, c->stream>>>(which == RAFEM_SYS_V ? c->instV : c->instT, c->n_inst, c->bar, which, c->stats, c->istats, 0);
    CK(cudaGetLastError());
    return finish(c, stats, false);
}

int rafem_solve_step(rafem_ctx* c, rafem_step_stats* stats) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    if (c->prm.n_corrector <= 1 && !c->mono) {
        CK(c->tracing ? enqueue_step_traced(c) : enqueue_step(c));
        const int s = finish(c, stats, false);
        const int t = tape_record(c, c->step);
        return t != RAFEM_OK ? t : s;
    }
    // fixed-point corrector passes: sigma at the newest T iterate, mass term at T^n (device-side loop)
    CK(launch_corrector_step(c));
    return finish(c, stats, false);
}

int rafem_step_host(rafem_ctx* c, const double* T_in, const double* V_in, double* T_out, double* V_out,
                    rafem_step_stats* stats) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    const size_t nb = (size_t)c->N * sizeof(double);
    if (c->prm.n_corrector > 1 || c->mono || c->tracing) {
        // corrector loop or traced step: the copies in sequence around the step
        if (T_in) CK(cudaMemcpyAsync(c->T, T_in, nb, cudaMemcpyHostToDevice, c->stream));
        if (V_in) CK(cudaMemcpyAsync(c->V, V_in, nb, cudaMemcpyHostToDevice, c->stream));
        const int s = rafem_solve_step(c, stats);
        if (s < 0) return s;
        if (T_out) CK(cudaMemcpyAsync(T_out, c->T, nb, cudaMemcpyDeviceToHost, c->stream));
        if (V_out) CK(cudaMemcpyAsync(V_out, c->V, nb, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        return s;
    }
    if (!c->io_stream) {
        CK(cudaStreamCreateWithFlags(&c->io_stream, cudaStreamNonBlocking));
        for (cudaEvent_t& e : c->io_ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const StepIO io{T_in, V_in, T_out, V_out};
    const void* key[4] = {T_in, V_in, T_out, V_out};
    if (!std::equal(key, key + 4, c->io_key)) {
        if (c->io_graph) cudaGraphExecDestroy(c->io_graph);
        c->io_graph = nullptr;
        c->io_graph_failed = false;
        std::copy(key, key + 4, c->io_key);
    }
    if (!c->io_graph && !c->io_graph_failed) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t e1 = enqueue_step_io(c, &io);
            const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
            if (e1 != cudaSuccess || e2 != cudaSuccess || !g || cudaGraphInstantiate(&c->io_graph, g, 0) != cudaSuccess)
                c->io_graph = nullptr;
            if (g) cudaGraphDestroy(g);
        }
        if (!c->io_graph) {
            c->io_graph_failed = true;  // e.g. pageable host buffers: direct launches
            cudaGetLastError();
        }
    }
    if (c->io_graph)
        CK(cudaGraphLaunch(c->io_graph, c->stream));
    else
        CK(enqueue_step_io(c, &io));
    const int s = finish(c, stats, false);
    const int t = tape_record(c, c->step);
    return t != RAFEM_OK ? t : s;
}

int rafem_run(rafem_ctx* c, int32_t n_steps, rafem_step_stats* last) {
    if (!c || n_steps < 0) return RAFEM_ERR_BAD_INPUT;
    if (n_steps == 0) return finish(c, last, true);
    k_set_step<<<1, 1, 0, c->stream>>>(c->stats, (long long)c->step);
    CK(cudaGetLastError());
    if (c->prm.n_corrector > 1 || c->mono) {
        for (int i = 0; i < n_steps; ++i) CK(launch_corrector_step(c));
        return finish(c, last, true);
    }
    const int64_t s0 = c->step;
    for (int i = 0; i < n_steps; ++i) {
        CK(launch_step(c));
        const int t = tape_record(c, s0 + i + 1);
        if (t != RAFEM_OK) return t;
    }
    return finish(c, last, true);
}

int rafem_get_field(rafem_ctx* c, int which, double* dst, int on_device) {
    if (!c || !dst || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    const double* src = which == RAFEM_SYS_V ? c->V : c->T;
    if (c->tracing) {
        for (int i = 0; i < 2; ++i)
            if (!c->ev[i]) CK(cudaEventCreate(&c->ev[i]));
        nvtxRangePushA("memcpyD2H");
        CK(cudaEventRecord(c->ev[0], c->stream));
    }
    CK(cudaMemcpyAsync(dst, src, c->N * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       c->stream));
    if (c->tracing) CK(cudaEventRecord(c->ev[1], c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->tracing) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        c->trace.ms_memcpy_d2h += ms;
        nvtxRangePop();
    }
    return RAFEM_OK;
}

int rafem_set_state(rafem_ctx* c, const double* T, const double* V, int on_device, int64_t step) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    c->tape_every = 0;
    cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->tracing) {
        for (int i = 0; i < 2; ++i)
            if (!c->ev[i]) CK(cudaEventCreate(&c->ev[i]));
        nvtxRangePushA("memcpyH2D");
        CK(cudaEventRecord(c->ev[0], c->stream));
    }
    if (T) CK(cudaMemcpyAsync(c->T, T, c->N * sizeof(double), kind, c->stream));
    if (V) CK(cudaMemcpyAsync(c->V, V, c->N * sizeof(double), kind, c->stream));
    if (c->tracing) {
        CK(cudaEventRecord(c->ev[1], c->stream));
        CK(cudaStreamSynchronize(c->stream));
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]);
        c->trace.ms_memcpy_h2d += ms;
        nvtxRangePop();
    }
    const bool continuing = step == c->step;
    c->step = step;
    k_set_step<<<1, 1, 0, c->stream>>>(c->stats, (long long)step);
    CK(cudaGetLastError());
    if (!continuing) {
        k_reset_hist<<<1, 1, 0, c->stream>>>(c->stats);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

int rafem_reorder_rcm(int32_t n_nodes, int32_t n_tets, const int32_t* tets, int32_t* perm) {
    if (!tets || !perm || n_nodes < 1 || n_tets < 1) return RAFEM_ERR_BAD_INPUT;
    for (int64_t q = 0; q < 4LL * n_tets; ++q)
        if (tets[q] < 0 || tets[q] >= n_nodes) return RAFEM_ERR_BAD_INPUT;
    try {
        std::vector<int32_t> p;
        reorder_rcm(n_nodes, n_tets, tets, p);
        std::copy(p.begin(), p.end(), perm);
    } catch (const std::bad_alloc&) {
        return RAFEM_ERR_OOM;
    }
    return RAFEM_OK;
}

int rafem_pattern_info(rafem_ctx* c, int32_t* n_rows, int64_t* nnz, int32_t* n_colors) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    if (n_rows) *n_rows = c->N;
    if (nnz) *nnz = c->nnz;
    if (n_colors) *n_colors = c->n_colors;
    return RAFEM_OK;
}

int rafem_batch_create(int32_t n, const rafem_mesh* const* meshes, const rafem_params* prm, void* stream,
                       rafem_ctx** out) {
    if (!out) return RAFEM_ERR_BAD_INPUT;
    *out = nullptr;
    if (!meshes || !prm || n < 1 || n > RAFEM_MAX_BATCH) return RAFEM_ERR_BAD_INPUT;
    // the union mesh: instance i's nodes start at off[i] (a multiple of 32); the nodes between instances are
    // isolated, Dirichlet in both systems, and touched by no element
    std::vector<int32_t> off(n + 1, 0);
    int64_t E = 0;
    for (int i = 0; i < n; ++i) {
        const rafem_mesh* m = meshes[i];
        if (!m || !m->coords || !m->tets || !m->bc_V || !m->g_V || !m->bc_T || !m->g_T || !m->sigma0 || !m->k ||
            m->n_nodes < 4 || m->n_tets < 1)
            return RAFEM_ERR_BAD_INPUT;
        const int64_t next = off[i] + ((int64_t)m->n_nodes + SELL_C - 1) / SELL_C * SELL_C;
        if (next > INT32_MAX / 2) return RAFEM_ERR_BAD_INPUT;
        off[i + 1] = (int32_t)next;
        E += m->n_tets;
    }
    if (E > INT32_MAX / 16) return RAFEM_ERR_BAD_INPUT;
    const int32_t N = off[n];
    std::vector<double> xyz(3 * (size_t)N, 0.0), gV(N, 0.0), gT(N, prm->T_a), s0, kk;
    std::vector<uint8_t> bV(N, 1), bT(N, 1);
    std::vector<int32_t> tets;
    tets.reserve(4 * (size_t)E);
    s0.reserve(E);
    kk.reserve(E);
    for (int i = 0; i < n; ++i) {
        const rafem_mesh* m = meshes[i];
        const int32_t o = off[i];
        std::copy(m->coords, m->coords + 3 * (size_t)m->n_nodes, xyz.begin() + 3 * (size_t)o);
        std::copy(m->g_V, m->g_V + m->n_nodes, gV.begin() + o);
        std::copy(m->g_T, m->g_T + m->n_nodes, gT.begin() + o);
        std::copy(m->bc_V, m->bc_V + m->n_nodes, bV.begin() + o);
        std::copy(m->bc_T, m->bc_T + m->n_nodes, bT.begin() + o);
        for (int64_t q = 0; q < 4LL * m->n_tets; ++q) {
            const int32_t v = m->tets[q];
            if (v < 0 || v >= m->n_nodes) return RAFEM_ERR_BAD_INPUT;
            tets.push_back(v + o);
        }
        s0.insert(s0.end(), m->sigma0, m->sigma0 + m->n_tets);
        kk.insert(kk.end(), m->k, m->k + m->n_tets);
    }
    rafem_mesh u{N, (int32_t)E, xyz.data(), tets.data(), bV.data(), gV.data(), bT.data(), gT.data(), s0.data(),
                 kk.data()};
    rafem_ctx* c = nullptr;
    int s = validate_params(&u, prm);
    if (s != RAFEM_OK) return s;
    c = new (std::nothrow) rafem_ctx();
    if (!c) return RAFEM_ERR_OOM;
    try {
        s = create_impl(&u, prm, stream, c, n, off);
    } catch (const std::bad_alloc&) {
        s = RAFEM_ERR_OOM;
    }
    if (s != RAFEM_OK) {
        rafem_destroy(c);
        return s;
    }
    *out = c;
    return RAFEM_OK;
}

int rafem_batch_info(rafem_ctx* c, int32_t* n_inst, int32_t* node_offsets) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    if (n_inst) *n_inst = c->n_inst;
    if (node_offsets) std::copy(c->inst_node_off.begin(), c->inst_node_off.end(), node_offsets);
    return RAFEM_OK;
}

int rafem_batch_stats(rafem_ctx* c, rafem_step_stats* per_instance) {
    if (!c || !per_instance) return RAFEM_ERR_BAD_INPUT;
    CK(cudaMemcpyAsync(per_instance, c->istats, c->n_inst * sizeof(rafem_step_stats), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

int rafem_batch_run(rafem_ctx* c, int32_t n_steps, rafem_step_stats* per_instance) {
    if (!c || n_steps < 0) return RAFEM_ERR_BAD_INPUT;
    const int s = rafem_run(c, n_steps, nullptr);
    if (s < 0 || !per_instance) return s;
    const int q = rafem_batch_stats(c, per_instance);
    return q != RAFEM_OK ? q : s;
}

int rafem_reset(rafem_ctx* c) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    c->tape_every = 0;
    const int N = c->N;
    k_init_fields<<<(N + 255) / 256, 256, 0, c->stream>>>(N, c->prm.T_a, c->bcT, c->gT, c->bcV, c->gV, c->T, c->V);
    CK(cudaGetLastError());
    for (double* h : {c->T_hist, c->V_hist, c->T_hist2, c->V_hist2, c->T_hist3, c->V_hist3})
        CK(cudaMemsetAsync(h, 0, N * sizeof(double), c->stream));
    if (c->proj_D) CK(cudaMemsetAsync(c->proj_D, 0, (size_t)proj_stride(c->proj_k) * N * sizeof(double), c->stream));
    CK(cudaMemsetAsync(c->istats, 0, c->n_inst * sizeof(rafem_step_stats), c->stream));
    CK(cudaMemsetAsync(c->stats, 0, sizeof(StatsDev), c->stream));
    c->step = 0;
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

namespace {

__global__ void k_widen(int n, const float* __restrict__ in, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

__global__ void k_narrow(int n, const double* __restrict__ in, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

// Where a parameter array comes from: host FP64, device FP64 or device FP32.
enum ParamSrc { SRC_HOST64 = 0, SRC_DEV64 = 1, SRC_DEV32 = 2 };

// Stage one parameter array into p_tmpE (FP64, mesh element order).
cudaError_t stage_param(rafem_ctx* c, const void* src, int kind) {
    const int E = c->E;
    if (kind == SRC_DEV32) {
        k_widen<<<(E + 255) / 256, 256, 0, c->stream>>>(E, static_cast<const float*>(src), c->p_tmpE);
        return cudaGetLastError();
    }
    return cudaMemcpyAsync(c->p_tmpE, src, E * sizeof(double),
                           kind == SRC_DEV64 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream);
}

int set_params_impl(rafem_ctx* c, const void* sigma0, const void* k, int kind) {
    if (!c || (!sigma0 && !k)) return RAFEM_ERR_BAD_INPUT;
    const int E = c->E;
    if (kind == SRC_HOST64) {
        for (const void* q : {sigma0, k})
            if (q)
                for (int e = 0; e < E; ++e)
                    if (!std::isfinite(static_cast<const double*>(q)[e])) return RAFEM_ERR_NONFINITE;
    }
    if (!c->p_tmpE) CK(dalloc(c, &c->p_tmpE, E));
    c->tape_every = 0;
    cudaStream_t st = c->stream;
    if (sigma0) {
        CK(stage_param(c, sigma0, kind));
        CK(launch_permute(E, c->e_order, c->p_tmpE, c->e_sig0, 0, st));
        if (c->dw)
            CK(launch_fill_dw(c->gdw, c->gather_nc, c->gd.celem, c->gather_cg, c->el, c->prm.rho_c / c->prm.dt, st));
        else if (c->gather)
            CK(launch_fill_cval(c->gather_nc, c->gd.celem, c->gather_cg, c->e_sig0, c->e_G, E,
                                const_cast<double*>(c->gd.cval), st));
    }
    if (k) {
        CK(stage_param(c, k, kind));
        CK(launch_permute(E, c->e_order, c->p_tmpE, c->e_k, 0, st));
        // constant thermal matrix and rhs part: every free slot is stored by its first writer, Dirichlet rows
        // keep the identity; the constant rhs accumulates and restarts from zero
        CK(cudaMemsetAsync(c->bTc, 0, c->N * sizeof(double), st));
        const double c_matrix = c->prm.rho_c / c->prm.dt + c->prm.perf;
        for (int q = 0; q < c->n_colors; ++q)
            CK(launch_assemble_T(c->el, c->color_off[q], c->color_off[q + 1], c->bcT, c->gT, c_matrix,
                                 c->prm.perf * c->prm.T_a, c->valsT, c->valsT32, c->bTc, c->prm.lift, c->e_clist, st));
        if (c->ilu) CK(ilu_refactor(c, RAFEM_SYS_T, st));
        if (c->mg.cab) CK(launch_coupled_fill(c->mg, c->gd, c->gather_nc, c->N, c->rp, c->diag, c->el, c_matrix, false, st));
    }
    CK(cudaStreamSynchronize(st));
    return RAFEM_OK;
}

}  // namespace

int rafem_set_params(rafem_ctx* c, const double* sigma0, const double* k, int on_device) {
    return set_params_impl(c, sigma0, k, on_device ? SRC_DEV64 : SRC_HOST64);
}

int rafem_set_params_device(rafem_ctx* c, const float* sigma0, const float* k) {
    return set_params_impl(c, sigma0, k, SRC_DEV32);
}

int rafem_precond_info(rafem_ctx* c, int32_t* n_levels, int32_t* padded_rows, int64_t* nnz_stored, int32_t* order,
                       int64_t* factor_stored, int32_t* column_bytes) {
    if (!c || !c->ilu) return RAFEM_ERR_BAD_INPUT;
    if (n_levels) *n_levels = c->il.n_levels;
    if (padded_rows) *padded_rows = c->il.Np;
    if (nnz_stored) *nnz_stored = c->il.nnz;
    if (factor_stored) *factor_stored = c->ir[0].nL + c->ir[0].nU;
    if (column_bytes) *column_bytes = c->ir[0].patterns ? 0 : 4;
    if (order) {
        int k = 0;
        for (int32_t o : c->ilu_perm)
            if (o >= 0) order[k++] = o;
    }
    return RAFEM_OK;
}

int rafem_get_precond(rafem_ctx* c, int which, double* factors) {
    if (!c || !c->ilu || !factors || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    std::vector<double> F(c->il.nnz);
    CK(cudaMemcpyAsync(F.data(), which == RAFEM_SYS_V ? c->ilu_FV : c->ilu_FT, F.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (size_t q = 0; q < F.size(); ++q)
        if (c->ilu_pmap_csr[q] >= 0) factors[c->ilu_pmap_csr[q]] = F[q];
    return RAFEM_OK;
}

int rafem_precond_apply(rafem_ctx* c, int which, const double* r, double* z) {
    if (!c || !r || !z || r == z || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    if (c->ilu) {
        CK(launch_ilu_apply(c->il, which == RAFEM_SYS_V ? c->ilu_FV : c->ilu_FT,
                            which == RAFEM_SYS_V ? c->ilu_DV : c->ilu_DT, r, z, c->ir[0].r64, c->ir[0].z64, c->stream));
    } else {
        k_jacobi_apply<<<(c->N + 255) / 256, 256, 0, c->stream>>>(c->N, c->diag,
                                                                   which == RAFEM_SYS_V ? c->valsV : c->valsT, r, z);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

namespace {

// Everything that depends on the step size: the thermal matrix and its constant right-hand side, the node masses
// of the thermal right-hand side and the thermal ILU factors. The captured graphs are dropped because their
// kernels take rho_c/dt as an argument.
int apply_dt(rafem_ctx* c, double dt) {
    c->prm.dt = dt;
    cudaStream_t st = c->stream;
    CK(cudaMemsetAsync(c->bTc, 0, c->N * sizeof(double), st));
    const double c_matrix = c->prm.rho_c / dt + c->prm.perf;
    for (int q = 0; q < c->n_colors; ++q)
        CK(launch_assemble_T(c->el, c->color_off[q], c->color_off[q + 1], c->bcT, c->gT, c_matrix,
                             c->prm.perf * c->prm.T_a, c->valsT, c->valsT32, c->bTc, c->prm.lift, c->e_clist, st));
    if (c->ilu) CK(ilu_refactor(c, RAFEM_SYS_T, st));
    if (c->gd.mT) CK(launch_node_mass(c->gd, c->N, c->e_vol, c->prm.rho_c / dt, st));
    if (c->dw) CK(launch_fill_dw(c->gdw, 0, nullptr, nullptr, c->el, c->prm.rho_c / dt, st));
    if (c->mg.cab) CK(launch_coupled_fill(c->mg, c->gd, c->gather_nc, c->N, c->rp, c->diag, c->el, c_matrix, false, st));
    drop_graphs(c);
    return RAFEM_OK;
}

}  // namespace

int rafem_graph_info(rafem_ctx* c, int32_t* step_graph, int32_t* corrector_graph, int32_t* step_kernels) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    if (step_kernels) *step_kernels = c->graph ? c->graph_kernels : 0;
    if (step_graph) *step_graph = c->graph ? 1 : (c->graph_failed ? 0 : -1);
    if (corrector_graph) *corrector_graph = c->corr_graph ? 1 : (c->corr_graph_failed ? 0 : -1);
    return RAFEM_OK;
}

int rafem_set_dt(rafem_ctx* c, double dt) {
    if (!c || !(dt > 0) || !std::isfinite(dt)) return RAFEM_ERR_BAD_INPUT;
    c->tape_every = 0;
    const int s = apply_dt(c, dt);
    if (s != RAFEM_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

int rafem_set_wait_limit(rafem_ctx* c, int64_t limit_ns, int32_t missing_arrivals) {
    if (!c || missing_arrivals < 0 || missing_arrivals > 1024) return RAFEM_ERR_BAD_INPUT;
    c->wait_ns = limit_ns > 0 ? (long long)limit_ns : kDefaultWaitNs;
    c->wait_missing = missing_arrivals;
    drop_graphs(c);  // the solver launches carry both as arguments
    return RAFEM_OK;
}

int rafem_set_tol(rafem_ctx* c, double tol, double inner_tol) {
    if (!c || !(tol > 0) || !std::isfinite(tol) || !(inner_tol < 1) || std::isnan(inner_tol)) return RAFEM_ERR_BAD_INPUT;
    c->prm.tol = tol;
    if (inner_tol > 0) c->prm.inner_tol = inner_tol;
    drop_graphs(c);  // the solver launches carry the tolerances as arguments
    return RAFEM_OK;
}

int rafem_advance(rafem_ctx* c, double duration, double dt_min, rafem_advance_stats* out) {
    if (!c || !(duration > 0) || !std::isfinite(duration) || !(dt_min > 0)) return RAFEM_ERR_BAD_INPUT;
    c->tape_every = 0;
    cudaStream_t st = c->stream;
    const size_t nb = (size_t)c->N * sizeof(double);
    const bool corrector = c->prm.n_corrector > 1 || c->mono;
    double t = 0.0, dt = c->prm.dt;
    int32_t accepted = 0, rejected = 0, passes = 0;
    k_set_step<<<1, 1, 0, st>>>(c->stats, (long long)c->step);
    CK(cudaGetLastError());
    while (t < duration * (1.0 - 1e-12)) {
        const double dt_step = std::min(dt, duration - t);
        if (dt_step != c->prm.dt) {
            const int s = apply_dt(c, dt_step);
            if (s != RAFEM_OK) return s;
        }
        CorrDev h{0, 1, 0.0};
        if (corrector) {
            CK(cudaMemcpyAsync(c->V_old, c->V, nb, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c->stats_save, c->stats, sizeof(StatsDev), cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c->istats_save, c->istats, c->n_inst * sizeof(rafem_step_stats),
                               cudaMemcpyDeviceToDevice, st));
            CK(launch_corrector_step(c));
            CK(cudaMemcpyAsync(&h, c->corr, sizeof(h), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        } else {
            CK(launch_step(c));
        }
        if (h.converged || dt_step * 0.5 < dt_min) {
            t += dt_step;
            ++accepted;
            passes += h.pass;
        } else {
            // not accepted: back to the state at the start of the step, retried with half the step size
            CK(cudaMemcpyAsync(c->T, c->T_old, nb, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c->V, c->V_old, nb, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c->stats, c->stats_save, sizeof(StatsDev), cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(c->istats, c->istats_save, c->n_inst * sizeof(rafem_step_stats),
                               cudaMemcpyDeviceToDevice, st));
            dt = dt_step * 0.5;
            ++rejected;
        }
    }
    if (c->prm.dt != dt) {  // keep the (possibly halved) step size, not the shortened last step
        const int s = apply_dt(c, dt);
        if (s != RAFEM_OK) return s;
    }
    rafem_step_stats last;
    const int s = finish(c, &last, true);
    if (out) {
        out->status = s;
        out->accepted = accepted;
        out->rejected = rejected;
        out->passes = passes;
        out->dt = dt;
        out->time = t;
    }
    return s;
}

int rafem_tape_begin(rafem_ctx* c, int32_t checkpoint_every) {
    if (!c || checkpoint_every < 1 || c->prm.n_corrector != 1 || c->prm.lift != RAFEM_LIFT_SYMMETRIC || c->mono)
        return RAFEM_ERR_BAD_INPUT;
    c->tape_every = 0;
    c->n_ckpt = 0;
    const int s = tape_save(c, 0);
    if (s != RAFEM_OK) return s;
    c->tape_every = checkpoint_every;
    c->tape_origin = c->step;
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

namespace {

// Workspace of the adjoint, and the node incidence + nodal mass when the assembly mode did not build them.
int ensure_adjoint(rafem_ctx* c) {
    const int N = c->N, E = c->E;
    if (!c->gd.ioff) {
        std::vector<int32_t> nodes_soa(4 * (size_t)E), i_off, i_cnt, i_elem;
        CK(cudaMemcpyAsync(nodes_soa.data(), c->e_nodes, nodes_soa.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        build_incidence(N, E, nodes_soa, i_off, i_cnt, i_elem);
        int32_t *ioff, *icnt, *ielem;
        double* mT;
        CK(dalloc(c, &ioff, i_off.size()));
        CK(dalloc(c, &icnt, i_cnt.size()));
        CK(dalloc(c, &ielem, i_elem.size()));
        CK(dalloc(c, &mT, N));
        CK(cudaMemcpyAsync(ioff, i_off.data(), i_off.size() * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(icnt, i_cnt.data(), i_cnt.size() * 4, cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(ielem, i_elem.data(), i_elem.size() * 4, cudaMemcpyHostToDevice, c->stream));
        c->gd.ioff = ioff;
        c->gd.icnt = icnt;
        c->gd.ielem = ielem;
        c->gd.mT = mT;
        CK(launch_node_mass(c->gd, N, c->e_vol, c->prm.rho_c / c->prm.dt, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    if (!c->adj_ready) {
        CK(dalloc(c, &c->a_lam, N));
        CK(dalloc(c, &c->a_mu, N));
        CK(dalloc(c, &c->a_nu, N));
        CK(dalloc(c, &c->a_h, N));
        CK(dalloc(c, &c->a_dv, N));
        CK(dalloc(c, &c->a_ew4, 4 * (size_t)E));
        CK(dalloc(c, &c->a_w, E));
        CK(dalloc(c, &c->a_gs, E));
        CK(dalloc(c, &c->a_gk, E));
        CK(dalloc(c, &c->a_count, 4));
        for (double** v : {&c->a_mu1, &c->a_mu2, &c->a_nu1, &c->a_nu2}) CK(dalloc(c, v, N));
        char* live = nullptr;
        CK(dalloc(c, &live, state_bytes(c)));
        c->ckpt_live = live;
        if (!c->p_tmpE) CK(dalloc(c, &c->p_tmpE, E));
        c->adj_ready = true;
    }
    if (c->seg_cap < c->tape_every) {
        CK(dalloc(c, &c->a_segT, (size_t)(c->tape_every + 1) * N));
        CK(dalloc(c, &c->a_segV, (size_t)c->tape_every * N));
        c->seg_cap = c->tape_every;
    }
    return RAFEM_OK;
}

int merge_status(int a, int b) {
    if (a < 0 || b < 0) return std::min(a, b);
    return std::max(a, b);
}

}  // namespace

int rafem_adjoint(rafem_ctx* c, const double* dL_dT, const double* dL_dV, int in_on_device, double* dL_dsigma0,
                  double* dL_dk, double* dL_dT0, int out_on_device, rafem_adjoint_stats* out) {
    if (!c || !dL_dT || c->tape_every <= 0 || out_on_device < 0 || out_on_device > 2) return RAFEM_ERR_BAD_INPUT;
    const auto t_start = std::chrono::steady_clock::now();
    const int64_t nsteps = c->step - c->tape_origin;
    const int every = c->tape_every;
    const int64_t n_seg = (nsteps + every - 1) / every;
    if (nsteps < 0 || nsteps > INT32_MAX || (size_t)n_seg > c->n_ckpt) return RAFEM_ERR_INTERNAL;
    {
        const int s = ensure_adjoint(c);
        if (s != RAFEM_OK) return s;
    }
    const int N = c->N, E = c->E;
    const size_t nb = (size_t)N * sizeof(double);
    cudaStream_t st = c->stream;
    const cudaMemcpyKind in_kind = in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double alpha = c->prm.alpha_sigma, c_mass = c->prm.rho_c / c->prm.dt;
    CK(cudaMemsetAsync(c->a_gs, 0, E * sizeof(double), st));
    CK(cudaMemsetAsync(c->a_gk, 0, E * sizeof(double), st));
    CK(cudaMemsetAsync(c->a_mu, 0, nb, st));
    CK(cudaMemsetAsync(c->a_nu, 0, nb, st));
    CK(cudaMemsetAsync(c->a_count, 0, 4 * sizeof(int32_t), st));
    CK(cudaMemcpyAsync(c->a_h, dL_dT, nb, in_kind, st));
    if (dL_dV) {
        CK(cudaMemcpyAsync(c->a_lam, dL_dV, nb, in_kind, st));
        CK(launch_mask(N, c->bcV, c->a_lam, c->a_dv, st));
    }
    int fwd_status = RAFEM_OK;
    if (nsteps == 0) {
        CK(cudaMemcpyAsync(c->a_lam, c->a_h, nb, cudaMemcpyDeviceToDevice, st));
    } else {
        CK(launch_mask(N, c->bcT, c->a_h, c->a_lam, st));
        CK(state_copy(c, c->ckpt_live, true));
        const int64_t live_step = c->step;
        int64_t done = 0;  // backward steps taken (history available to the extrapolation)
        const int saved_every = c->tape_every;
        c->tape_every = 0;  // the recomputation must not write checkpoints
        for (int64_t seg = n_seg - 1; seg >= 0; --seg) {
            const int64_t b0 = seg * every, b1 = std::min<int64_t>(b0 + every, nsteps);
            const int L = (int)(b1 - b0);
            CK(state_copy(c, c->ckpt[seg], false));
            CK(cudaMemcpyAsync(c->a_segT, c->T, nb, cudaMemcpyDeviceToDevice, st));
            for (int j = 0; j < L; ++j) {
                CK(launch_step(c));
                CK(cudaMemcpyAsync(c->a_segT + (size_t)(j + 1) * N, c->T, nb, cudaMemcpyDeviceToDevice, st));
                CK(cudaMemcpyAsync(c->a_segV + (size_t)j * N, c->V, nb, cudaMemcpyDeviceToDevice, st));
            }
            k_fold_worst<<<1, 1, 0, st>>>(c->stats, c->a_count + 3);
            CK(cudaGetLastError());
            for (int j = L - 1; j >= 0; --j) {
                const int64_t n = b0 + j;
                const double* Tn = c->a_segT + (size_t)j * N;
                const double* T1 = c->a_segT + (size_t)(j + 1) * N;
                const double* V1 = c->a_segV + (size_t)j * N;
                // initial guesses extrapolated along the backward sweep (the forward predictor's order, at most 2)
                const int q = (int)std::min<int64_t>(std::min(c->prm.predictor, 2), done);
                CK(launch_adj_extrapolate(N, c->a_mu, c->a_mu1, c->a_mu2, q, st));
                CK(enqueue_solve(c, RAFEM_SYS_T, c->a_lam, c->a_mu));
                CK(launch_adj_count(c->instT, c->n_inst, c->bar, c->a_count, 1, st));
                CK(enqueue_assemble(c, RAFEM_SYS_V, Tn, Tn));
                CK(launch_adj_h(c->el, c->gd, N, Tn, V1, c->a_mu, alpha, c->bcV,
                                (dL_dV && n == nsteps - 1) ? c->a_dv : nullptr, c->a_ew4, c->a_h, st));
                CK(launch_adj_extrapolate(N, c->a_nu, c->a_nu1, c->a_nu2, q, st));
                CK(enqueue_solve(c, RAFEM_SYS_V, c->a_h, c->a_nu));
                CK(launch_adj_count(c->instV, c->n_inst, c->bar, c->a_count, 0, st));
                CK(launch_adj_g(c->el, c->gd, N, Tn, V1, T1, c->a_mu, c->a_nu, alpha, c_mass, c->bcT, n != 0,
                                c->a_gs, c->a_gk, c->a_w, c->a_lam, st));
                ++done;
            }
        }
        CK(state_copy(c, c->ckpt_live, false));
        c->step = live_step;
        c->tape_every = saved_every;
    }
    // outputs (gradients back in mesh element order); out_on_device 2: element gradients as device floats
    const cudaMemcpyKind out_kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    double* grads_dst[2] = {dL_dsigma0, dL_dk};
    const double* grads_src[2] = {c->a_gs, c->a_gk};
    for (int q = 0; q < 2; ++q) {
        if (!grads_dst[q]) continue;
        if (out_on_device == 1) {
            CK(launch_permute(E, c->e_order, grads_src[q], grads_dst[q], 1, st));
            continue;
        }
        CK(cudaStreamSynchronize(st));  // p_tmpE is reused
        CK(launch_permute(E, c->e_order, grads_src[q], c->p_tmpE, 1, st));
        if (out_on_device == 2) {
            k_narrow<<<(E + 255) / 256, 256, 0, st>>>(E, c->p_tmpE, reinterpret_cast<float*>(grads_dst[q]));
            CK(cudaGetLastError());
        } else {
            CK(cudaMemcpyAsync(grads_dst[q], c->p_tmpE, E * sizeof(double), out_kind, st));
        }
    }
    if (dL_dT0) CK(cudaMemcpyAsync(dL_dT0, c->a_lam, nb, out_kind, st));
    int32_t cnt[4];
    CK(cudaMemcpyAsync(cnt, c->a_count, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int adj_status = cnt[2];
    fwd_status = cnt[3];
    if (out) {
        out->status = adj_status;
        out->forward_status = fwd_status;
        out->steps = (int32_t)nsteps;
        out->segments = (int32_t)n_seg;
        out->iters_V = cnt[0];
        out->iters_T = cnt[1];
        out->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    }
    return merge_status(adj_status, fwd_status);
}

int rafem_set_schedule(rafem_ctx* c, int32_t rows_per_tile) {
    if (!c || rows_per_tile < 0) return RAFEM_ERR_BAD_INPUT;
    return build_tiles(c, rows_per_tile);
}

int rafem_get_schedule(rafem_ctx* c, int32_t* rows_per_tile, int32_t* n_tiles, int32_t* grid) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    if (rows_per_tile) *rows_per_tile = c->rows_per_tile;
    if (n_tiles) *n_tiles = c->n_tiles;
    if (grid) *grid = c->grid;
    return RAFEM_OK;
}

int rafem_layout_info(rafem_ctx* c, int32_t* kernel_code, int64_t* nnz_stored, int32_t* column_bytes,
                      int32_t* assembly, int32_t* arith) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    if (kernel_code) *kernel_code = c->lanes;
    if (nnz_stored) *nnz_stored = c->nnz_store;
    if (column_bytes) *column_bytes = c->ci16 ? 2 : 4;
    if (assembly) *assembly = c->gather ? RAFEM_ASSEMBLY_GATHER : RAFEM_ASSEMBLY_COLOR;
    if (arith) *arith = c->dw ? RAFEM_ARITH_DW : RAFEM_ARITH_FP64;
    return RAFEM_OK;
}

int rafem_get_system(rafem_ctx* c, int which, int32_t* row_ptr, int32_t* col, double* vals, double* rhs) {
    if (!c || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    cudaStream_t st = c->stream;
    if (row_ptr) std::copy(c->h_rp.begin(), c->h_rp.end(), row_ptr);
    if (col) std::copy(c->h_col.begin(), c->h_col.end(), col);
    std::vector<double> store;
    if (vals) {
        store.resize(c->nnz_store);
        CK(cudaMemcpyAsync(store.data(), which == RAFEM_SYS_V ? c->valsV : c->valsT, c->nnz_store * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
    }
    if (rhs)
        CK(cudaMemcpyAsync(rhs, which == RAFEM_SYS_V ? c->bV : c->bT, c->N * sizeof(double), cudaMemcpyDeviceToHost,
                           st));
    CK(cudaStreamSynchronize(st));
    if (vals) {
        if (c->sell)
            for (int64_t k = 0; k < c->nnz; ++k) vals[k] = store[c->h_map[k]];
        else
            std::copy(store.begin(), store.end(), vals);
    }
    return RAFEM_OK;
}

int rafem_get_coupled_system(rafem_ctx* c, double* blocks, double* residual) {
    if (!c || !c->mono) return RAFEM_ERR_BAD_INPUT;
    CK(cudaMemcpyAsync(c->T_old, c->T, c->N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    cudaStream_t st = c->stream;
    CK(enqueue_coupled_assembly(c));
    std::vector<double> v4(4 * (size_t)c->nnz_store);
    CK(cudaMemcpyAsync(v4.data(), c->m_vals4, v4.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (residual) CK(cudaMemcpyAsync(residual, c->m_R, 2 * (size_t)c->N * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (blocks)
        for (int64_t q = 0; q < c->nnz; ++q) {
            const size_t pos = 4 * (size_t)(c->sell ? c->h_map[q] : q);
            for (int k = 0; k < 4; ++k) blocks[4 * q + k] = v4[pos + k];
        }
    return RAFEM_OK;
}

int rafem_spmv(rafem_ctx* c, int which, const double* x, double* y) {
    if (!c || !x || !y || (which != RAFEM_SYS_V && which != RAFEM_SYS_T)) return RAFEM_ERR_BAD_INPUT;
    CK(launch_spmv64(c->N, c->sell ? 1 : 0, c->rp, c->ci, which == RAFEM_SYS_V ? c->valsV : c->valsT, x, y,
                     c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RAFEM_OK;
}

int rafem_set_tracing(rafem_ctx* c, int enable) {
    if (!c) return RAFEM_ERR_BAD_INPUT;
    c->tracing = enable != 0;
    c->trace = rafem_trace{};
    return RAFEM_OK;
}

int rafem_get_trace(rafem_ctx* c, rafem_trace* out) {
    if (!c || !out) return RAFEM_ERR_BAD_INPUT;
    *out = c->trace;
    return RAFEM_OK;
}

}  // extern "C"
