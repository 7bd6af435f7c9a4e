// Internal declarations shared by the CUDA translation units of librafem (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/rafem.h"

namespace rafem {

// ------------------------------------------------------------------------------------------------------------
// Element data, SoA over the element storage order (colour-sorted for the colour scatter, by smallest node for
// the row-owner assembly). G holds the 10 distinct entries of
// vol_e * grad(phi_a) . grad(phi_b) in the order (00,11,22,33,01,02,03,12,13,23).
// ------------------------------------------------------------------------------------------------------------
struct ElemData {
    int E = 0;
    const int32_t* nodes = nullptr;   // [4][E]
    const int32_t* slots = nullptr;   // [16][E] slot codes (setup.h flags)
    const double* G = nullptr;        // [10][E]
    const double* vol = nullptr;      // [E]
    const double* sigma0 = nullptr;   // [E]
    const double* k = nullptr;        // [E]
};

// Row-owner assembly data (SELL-32 layout; see setup.h build_gather / build_incidence).
struct GatherData {
    const int32_t* goff = nullptr;   // [nnz_store/32] start of each (slice, column) contribution group
    const int32_t* gcnt = nullptr;   // [nnz_store/32] contributions per lane in the group
    const double* cval = nullptr;    // sigma0_e G_e[a][b] per contribution (0 for padding)
    const int32_t* celem = nullptr;  // element (sorted order) per contribution
    const int32_t* ioff = nullptr;   // [N/32] node -> element incidence, per slice
    const int32_t* icnt = nullptr;
    const int32_t* ielem = nullptr;  // 4 e + a (element, local vertex); -1 = padding
    double* ework = nullptr;         // [E] per-element factor (f_e, then w_e)
    double* mT = nullptr;            // [N] (rho_c/dt) sum vol/20
};

// Double-word (float pair) data of the gather assembly (assembly_dw.cu): the element constants, split once per
// context, and per-pass node copies of the fields.
struct GatherDw {
    float2* cval = nullptr;  // sigma0_e G_e[a][b] per contribution, as GatherData::cval
    float2* tq = nullptr;    // [7][E]: -sigma0_e G_e[ab] / 4 for the six edges, then (rho_c/dt) vol_e / 20
    float2* Ts = nullptr;    // [N] temperature of sigma(T)
    float2* To = nullptr;    // [N] temperature of the mass term (T^n)
    float2* V = nullptr;     // [N] potential
};
cudaError_t launch_fill_dw(const GatherDw& d, long long nc, const int32_t* celem, const uint8_t* cg,
                           const ElemData& el, double c_mass, cudaStream_t st);
// With D non-null the assembly also accumulates Y = A D (the lifted matrix times the projection basis, 4
// double-word entries per node) on free rows, when kin[0] > 0.
cudaError_t launch_assemble_V_gather_dw(const GatherData& gd, const GatherDw& d, int N, const int32_t* sp,
                                        const int32_t* sc, const int32_t* diag, const ElemData& el, const double* T,
                                        double alpha, const uint8_t* bc, const double* g, double* vals, float* vals32,
                                        double* b, int row_lift, const double* D, double* Y, const int32_t* kin,
                                        cudaStream_t st);
cudaError_t launch_rhs_T_gather_dw(const GatherData& gd, const GatherDw& d, int N, const ElemData& el,
                                   const double* T_sigma, const double* T_old, const double* V, const uint8_t* bc,
                                   const double* g, const double* bconst, double alpha, double* b, cudaStream_t st);

// Launchers (assembly.cu). Every launcher only enqueues work on `st`.
cudaError_t launch_fill_cval(long long nc, const int32_t* celem, const uint8_t* cg, const double* sigma0,
                             const double* G, int E, double* cval, cudaStream_t st);
cudaError_t launch_assemble_V_gather(const GatherData& gd, int N, const int32_t* sp, const int32_t* sc,
                                     const int32_t* diag, const ElemData& el, const double* T, double alpha,
                                     const uint8_t* bc, const double* g, double* vals, float* vals32, double* b,
                                     int row_lift, cudaStream_t st);
cudaError_t launch_rhs_T_gather(const GatherData& gd, int N, const ElemData& el, const double* T_sigma,
                                const double* T_old, const double* V, const uint8_t* bc, const double* g,
                                const double* bconst, double alpha, double c_mass, double* b, cudaStream_t st);
cudaError_t launch_node_mass(const GatherData& gd, int N, const double* vol, double c_mass, cudaStream_t st);
cudaError_t launch_geometry(const ElemData& el, const double* xyz, double* G, double* vol, cudaStream_t st);
cudaError_t launch_init_rhs(int N, const uint8_t* bc, const double* g, const double* base, double* b,
                            cudaStream_t st);
cudaError_t launch_set_dirichlet_identity(int N, const uint8_t* bc, const int32_t* diag, double* vals,
                                          float* vals32, cudaStream_t st);
// A_V(sigma(T)) for elements [e0, e1) of one colour; lifted rhs contributions into b (row_lift: Dirichlet columns
// stay in the matrix, nothing moves to the rhs).
cudaError_t launch_assemble_V(const ElemData& el, int e0, int e1, const double* T, const uint8_t* bc,
                              const double* g, double alpha, double* vals, float* vals32, double* b, int row_lift,
                              cudaStream_t st);
// Constant thermal matrix c_mass*M + K_k for one colour; constant rhs part (perfusion + lift) into bconst. The
// colour's elements are positions [e0, e1) of `list` (storage indices in colour order), or storage indices
// [e0, e1) themselves when list is null.
cudaError_t launch_assemble_T(const ElemData& el, int e0, int e1, const uint8_t* bc, const double* g,
                              double c_matrix, double perf_Ta, double* vals, float* vals32, double* bconst,
                              int row_lift, const int32_t* list, cudaStream_t st);
// Thermal right-hand side for one colour: Joule source + (rho_c/dt) M T_old, free rows only.
cudaError_t launch_rhs_T(const ElemData& el, int e0, int e1, const double* T_sigma, const double* T_old,
                         const double* V, const uint8_t* bc, double alpha, double c_mass, double* b,
                         cudaStream_t st);
// y = A x in FP64 for either storage layout (sell = 1: SELL-32 slices sp/sc; sell = 0: CSR rp/ci).
cudaError_t launch_spmv64(int N, int sell, const int32_t* rp_or_sp, const int32_t* ci_or_sc, const double* A,
                          const double* x, double* y, cudaStream_t st);
cudaError_t launch_max_abs_diff(int N, const double* a, const double* b, double* out, cudaStream_t st);
// Monolithic coupled step: Jacobian blocks (4 per stored entry) and interleaved residual of the colour [e0, e1)
// (positions of `list`, or storage indices when null); Dirichlet rows; Newton update.
cudaError_t launch_coupled(const ElemData& el, int e0, int e1, const int32_t* list, const double* V, const double* T,
                           const double* T_old, double alpha, double c_dt, double perf, double T_a, double* vals4,
                           double* R, cudaStream_t st);
cudaError_t launch_coupled_dirichlet(int N, int sell, const int32_t* rp, const int32_t* diag, const uint8_t* bcV,
                                     const uint8_t* bcT, const double* gV, const double* gT, const double* V,
                                     const double* T, double* vals4, double* R, cudaStream_t st);
cudaError_t launch_newton_update(int N, const double* delta, double* V, double* T, cudaStream_t st);

// Row-owner assembly of the coupled Jacobian and residual (coupled_gather.cu), on the gather lists of GatherData.
struct CoupledGather {
    uint8_t* cab = nullptr;  // per contribution: 4 a + b (row vertex a, column vertex b of the element), 255 padding
    double* Gc = nullptr;    // per contribution: G_e[a][b] (0 for padding)
    double* tc = nullptr;    // [nnz_store] constant thermal block, unlifted: k G + (rho_c/dt + perf) M
    double2* rec = nullptr;  // [E][4] per element: {sigma, ds}, {-ds quad / 4, 0}, {(G V)_0, (G V)_1}, {(G V)_2, (G V)_3}
    double* rt = nullptr;    // [4 E] thermal residual contribution per (element, vertex), less tc T
};
// Gc (when geometry is set: once per context) and tc (again whenever k or rho_c/dt + perf = cm changes).
cudaError_t launch_coupled_fill(const CoupledGather& cg, const GatherData& gd, long long nc, int N, const int32_t* sp,
                                const int32_t* diag, const ElemData& el, double cm, bool geometry, cudaStream_t st);
// Every entry of vals4 (padding as zero) and of R is written: no clearing needed.
cudaError_t launch_coupled_gather(const CoupledGather& cg, const GatherData& gd, int N, const int32_t* sp,
                                  const int32_t* sc, const int32_t* diag, const ElemData& el, const double* V, const double* T,
                                  const double* T_old, double alpha, double c_dt, double perf, double T_a,
                                  const uint8_t* bcV, const uint8_t* bcT, const double* gV, const double* gT,
                                  double* vals4, double* R, cudaStream_t st);

// ------------------------------------------------------------------------------------------------------------
// Persistent Krylov solver (krylov.cu)
// ------------------------------------------------------------------------------------------------------------
struct InstState {
    double bb;          // ||b||^2 (FP64)
    double rr;          // latest ||r||^2 of the running (inner) iteration
    double rr0;         // mixed: FP64 ||r||^2 at the start of the current refinement
    double rr_in0;      // mixed: inner ||r32||^2 at the start of the current inner solve
    double gamma;       // mixed: inner gamma of the start vector
    double gamma_prev;  // (r, M^-1 r) of the previous iteration
    double alpha_prev;
    double alpha, beta;
    double relres;      // final FP64 relative residual
    int32_t iters;      // Krylov iterations (all refinements)
    int32_t refine;     // FP64 refinements done
    int32_t status;
    int32_t active;     // 1 while the instance still iterates
    int32_t first;      // 1 before the first iteration of a (inner) CG run
    int32_t outer;      // mixed: state of the refinement state machine
    int32_t mbuf;       // mixed: which m buffer holds M^-1 w of the current iteration
    int32_t breakdowns; // mixed: inner solves ended early by an FP32 curvature breakdown
    // mixed: FP32 coefficients of the inner iteration and its stopping threshold on ||r32||^2
    float alpha32, beta32, gprev32, aprev32, thr32, pad32;
};

// Number of per-tile partial sums a solver kernel writes (gamma, rr, delta, bb, rr64).
constexpr int kPartialQ = 5;

// Default wall-clock limit of every bounded device wait (grid barriers, copy slots): 5 s.
constexpr long long kDefaultWaitNs = 5000000000LL;

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int err;
    int n_active;       // instances still iterating (written by the last arriver)
    unsigned int pad[28];
};

// Enqueue the reset of a solver launch's barrier: counter at 0 - missing (missing > 0 only in tests: the first
// barrier then cannot complete and its waits run out), no error recorded.
cudaError_t launch_barrier_reset(GridBarrier* bar, int missing, cudaStream_t st);

struct SolveArgs {
    // matrix (lifted, fixed pattern): CSR (rp, ci) or SELL-32 (rp = slice pointers, ci = slice columns)
    int N;
    const int32_t* rp;
    const int32_t* ci;
    const int16_t* ci16;  // SELL-32 column deltas col - row (kernel code 2), when every delta fits 16 bits
    const int32_t* pat_off;   // kernel code 3: first offset of each slice's column pattern in pat_pool
    const int32_t* pat_pool;  // kernel code 3: the distinct slice patterns (column - row per slot)
    const double* A;
    const float* A32;
    const int32_t* diag;  // slot of the diagonal entry of each row
    // problem
    const double* b;
    double* x;
    const double* r0;        // b - A x for the starting x, computed by the predictor, or null (CG kernels read it in
    const int32_t* r0_ok;    // place of their first residual SpMV for instances i with r0_ok[i] > 0)
    // FP64 workspace
    double *r, *u, *w, *p, *s, *dinv;
    // FP32 workspace (mixed precision)
    float *r32, *u32, *w32, *p32, *s32, *d32, *dinv32;
    double *z, *q, *ma, *mb;  // pipelined CG: z = A q, q = M^-1 s, m = M^-1 w (double-buffered ma / mb)
    // work tiles: contiguous row ranges, each belonging to one instance
    int n_tiles;
    const int32_t* tile_r0;
    const int32_t* tile_r1;
    const int32_t* tile_inst;
    int n_inst;
    const int32_t* inst_t0;  // first tile of each instance
    const int32_t* inst_t1;  // one past its last tile
    InstState* inst;
    double* partial;         // [kPartialQ][n_tiles]
    GridBarrier* bar;
    // controls
    double tol, inner_tol;
    int max_iter, max_refine;
    long long spin_limit_ns;
    int bar_missing;         // testing: the barrier counter starts this many arrivals short (0 in normal use)
    const int* skip;         // when set and nonzero at launch, the solve does nothing (a finished outer iteration)
};

// Kernel code: 1 = SELL-32 with 32-bit columns, 2 = SELL-32 with 16-bit column deltas, 3 = SELL-32 whose slices
// share one column pattern (values streamed, no columns), 4/8/16/32 = CSR with that many lanes per row.
int krylov_max_blocks(int lanes, int precision, bool pipelined, int* block_threads);
cudaError_t launch_krylov(const SolveArgs& a, int lanes, int precision, bool pipelined, int grid, int block,
                          cudaStream_t st);

}  // namespace rafem

namespace rafem {

// ------------------------------------------------------------------------------------------------------------
// Differentiation form (adjoint.cu). gd must hold the node incidence (4 e + a entries) and mT.
// ------------------------------------------------------------------------------------------------------------
// h = sum over incident (e, a) of 2 s_e sigma_e (G_e V_e)_a (+ extra) on free rows of bcV, 0 on Dirichlet rows;
// ew4 is [4][E] scratch.
cudaError_t launch_adj_h(const ElemData& el, const GatherData& gd, int N, const double* Tn, const double* V,
                         const double* mu, double alpha, const uint8_t* bcV, const double* extra, double* ew4,
                         double* h, cudaStream_t st);
// gs += dL/dsigma0, gk += dL/dk of one step (sorted element order); lam = dL/dT^n (w is [E] scratch).
cudaError_t launch_adj_g(const ElemData& el, const GatherData& gd, int N, const double* Tn, const double* V,
                         const double* T1, const double* mu, const double* nu, double alpha, double c_mass,
                         const uint8_t* bcT, int zero_dirichlet, double* gs, double* gk, double* w, double* lam,
                         cudaStream_t st);
cudaError_t launch_mask(int N, const uint8_t* bc, const double* in, double* out, cudaStream_t st);
cudaError_t launch_permute(int n, const int32_t* perm, const double* in, double* out, int scatter, cudaStream_t st);
cudaError_t launch_adj_count(const InstState* inst, int n_inst, const GridBarrier* bar, int32_t* acc, int slot,
                             cudaStream_t st);
// x <- extrapolation of order q (0..2) from x (newest), h1, h2; history shifted (h2 <- h1 <- x).
cudaError_t launch_adj_extrapolate(int N, double* x, double* h1, double* h2, int q, cudaStream_t st);

}  // namespace rafem

namespace rafem {

// ------------------------------------------------------------------------------------------------------------
// ILU(0) preconditioner (ilu.cu): level-ordered permuted SELL-32 layout (setup.h IluHost) on the device.
// ------------------------------------------------------------------------------------------------------------
struct IluLayout {
    int Np = 0, n_levels = 0;
    long long nnz = 0;               // stored entries (with padding)
    const int32_t* lvl = nullptr;    // [n_levels + 1] (device)
    const int32_t* sp = nullptr;     // [Np/32 + 1]
    const int32_t* sc = nullptr;     // [nnz]
    const int32_t* pmap = nullptr;   // [nnz] source position in the system's value storage; -1 pad, -2 unit
    const uint8_t* rlen = nullptr;   // [Np]
    const uint8_t* dk = nullptr;     // [Np]
    const int32_t* perm = nullptr;   // [Np] original row, -1 dummy
    std::vector<int32_t> h_lvl;      // host copy of lvl
};


// ILU(0)-PCG streaming its matrices through the shared-memory ring (ilu_ring.cu): layouts of P A P^T, L and U
// (setup.h IluRingHost) on the device, the values of one system, and the solver workspace (shared by both
// systems of a context).
constexpr int kIluRingSlots = 8;  // partial-sum slots of the ring ILU solver, each [grid]
struct IluRingPartDev {
    const int32_t* sp = nullptr;
    const int32_t* sc = nullptr;
    const int32_t* pat_off = nullptr;
    const int32_t* pat_pool = nullptr;
    const int32_t* src = nullptr;   // position in the combined factor layout, -1 padding
};
struct IluRingDev {
    int Np = 0, n_levels = 0;
    bool patterns = false;          // all three layouts share one column pattern per slice
    const int32_t* lvl = nullptr;   // [n_levels + 1]
    const int32_t* perm = nullptr;  // [Np]
    IluRingPartDev A, L, U;
    long long nA = 0, nL = 0, nU = 0;
    double *A64 = nullptr, *L64 = nullptr, *U64 = nullptr;           // FP64 values (L, U: FP64 Krylov only)
    float *A32 = nullptr, *L32 = nullptr, *U32 = nullptr, *dinv32 = nullptr;  // mixed precision only
    double *xv = nullptr, *bv = nullptr, *r64 = nullptr, *z64 = nullptr, *p64 = nullptr, *q64 = nullptr;
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
    double* partial = nullptr;      // [kIluRingSlots][grid]
};
struct IluRingSolve {
    const IluRingDev* d;
    bool mixed;
    int N;
    const double* dinv64;           // 1 / u_ii (FP64, padded level order)
    const double* b;
    double* x;
    GridBarrier* bar;
    InstState* inst;
    double tol, inner_tol;
    int max_iter, max_refine;
    long long spin_limit_ns;
    int bar_missing;
};
int ilu_ring_max_blocks();
// Values of the ring layouts from the combined layout (Ap: the permuted system, F: its factors, dinv: 1 / u_ii).
cudaError_t launch_ilu_ring_split(const IluRingDev& d, const double* Ap, const double* F, const double* dinv,
                                  bool mixed, cudaStream_t st);
cudaError_t launch_ilu_ring(const IluRingSolve& s, int grid, cudaStream_t st);

// Ap = permuted values of `vals` (the system in its primary storage), F = ILU(0) factors of Ap, level by level,
// dinv = 1 / diag(U).
cudaError_t launch_ilu_refactor(const IluLayout& L, const double* vals, double* Ap, double* F, double* dinv,
                                cudaStream_t st);
// z = U^-1 L^-1 r (original ordering; rv, zv: [Np] scratch).
cudaError_t launch_ilu_apply(const IluLayout& L, const double* F, const double* dinv, const double* r, double* z,
                             double* rv, double* zv, cudaStream_t st);

}  // namespace rafem

namespace rafem {

// ------------------------------------------------------------------------------------------------------------
// Persistent Jacobi-BiCGSTAB, FP64, single instance, SELL-32 primary storage (bicgstab.cu).
// ------------------------------------------------------------------------------------------------------------
struct BicgArgs {
    int block = 1;                   // 1: scalar rows; 2: 2 x 2 block rows (A holds 4 values per stored entry,
                                     // vectors 2 values per row, block-Jacobi preconditioner)
    int N;
    const int32_t* sp;               // slice pointers
    const int32_t* sc;               // 32-bit columns (used when sc16 is null)
    const int16_t* sc16;             // 16-bit column deltas or null
    const int32_t* pat_off = nullptr;   // scalar rows: one column pattern per slice (kernel code 3), or null
    const int32_t* pat_pool = nullptr;
    const double* A;
    const int32_t* diag;             // storage position of each row's diagonal
    const double* b;
    double* x;                       // initial guess in, solution out
    double *r, *rh, *p, *ph, *v, *s, *sh, *t, *dinv;  // [N] workspace
    double* partial;                 // [bicgstab_partial_slots()][grid]
    GridBarrier* bar;
    InstState* inst;
    double tol;
    int max_iter;
    long long spin_limit_ns;
    int bar_missing;         // testing: the barrier counter starts this many arrivals short (0 in normal use)
    double* newton = nullptr;  // monolithic step: inexact-Newton forcing state (bicgstab.cu), else null
};
// block = 1 runs the ring kernel of bicgstab_ring.cu, block = 2 the block kernel of bicgstab.cu.
int bicgstab_max_blocks(int block);
int bicgstab_partial_slots();
cudaError_t launch_bicgstab(const BicgArgs& a, int grid, cudaStream_t st);
int bicgstab_ring_max_blocks();
int bicgstab_ring_partial_slots();
cudaError_t launch_bicgstab_ring(const BicgArgs& a, int grid, cudaStream_t st);

}  // namespace rafem

namespace rafem {

// ------------------------------------------------------------------------------------------------------------
// Persistent restarted GMRES(m), FP64, right Jacobi preconditioning, SELL-32 primary storage (gmres.cu).
// ------------------------------------------------------------------------------------------------------------
struct GmresArgs {
    int N, m;                        // rows, restart length (1..64): the longest cycle
    int m_min;                       // 0: every cycle has m steps; else cycles adapt between m_min and m
    int ld;                          // row stride of the basis: N rounded up to a multiple of 32
    const int32_t* sp;
    const int32_t* sc;
    const int16_t* sc16;
    const int32_t* pat_off;          // one column pattern per slice (kernel code 3), or null
    const int32_t* pat_pool;
    const double* A;
    const int32_t* diag;
    const double* b;
    double* x;
    double* V;                       // [m][ld] basis
    double *w0, *w1, *z, *dinv;      // [N]
    double* H;                       // [grid][(m + 1) m] Hessenberg matrix, one copy per block
    double* partial;                 // [gmres_partial_slots(m)][grid]
    GridBarrier* bar;
    InstState* inst;                 // iters = Arnoldi steps, refine = restart cycles
    double tol;
    int max_iter;
    long long spin_limit_ns;
    int bar_missing;         // testing: the barrier counter starts this many arrivals short (0 in normal use)
};
int gmres_max_blocks(int m);
int gmres_partial_slots(int m);
cudaError_t launch_gmres(const GmresArgs& a, int grid, cudaStream_t st);

}  // namespace rafem

namespace rafem {

// ------------------------------------------------------------------------------------------------------------
// Initial guess by A-orthogonal projection onto the last solutions (project.cu).
// ------------------------------------------------------------------------------------------------------------
constexpr int kProjChunk = 1024;  // rows per block of the projection passes
constexpr int kProjMax = 8;                                       // solutions in the basis, at most
constexpr int kProjDefault = 4;  // default: the best time to solution over a whole run (larger bases cost more
                                 // per step than they save once the solves take a few iterations)
constexpr int kProjQ = kProjMax * (kProjMax + 1) / 2 + kProjMax;  // Gram entries + right-hand sides, at most
// Entries per node of the basis arrays for a limit of k solutions (even, so that pairs load as 16 bytes).
inline int proj_stride(int k) { return k <= 2 ? 2 : (k <= 4 ? 4 : (k <= 6 ? 6 : 8)); }

struct ProjArgs {
    int n_tiles;
    int n_sub;                       // chunks of kProjChunk rows per tile (the largest tile's count)
    const int32_t* tile_r0;
    const int32_t* tile_r1;
    const int32_t* tile_inst;
    int n_inst;
    const int32_t* inst_t0;
    const int32_t* inst_t1;
    int sell;                        // 1: SELL-32 slice pointers in rp; 0: CSR row pointers
    const int32_t* rp;
    const int32_t* ci;
    const int16_t* ci16;             // 16-bit column deltas or null
    const double* A;                 // lifted SPD system (storage layout)
    const uint8_t* bc;               // Dirichlet rows
    const double* b;
    double* x;                       // x_n in, initial guess out
    int kmax;                        // basis size limit (1..kProjMax)
    double* D;                       // [N][proj_stride(kmax)] basis, 8-byte entries (FP64 or float pairs); the
                                     // previous call's basis on entry (the predictor's history)
    double* Y;                       // [N][proj_stride(kmax)] A D
    double* r0;                      // [N] out: b - A x of the guess (b - Y c; 0 on Dirichlet rows) where kout > 0
    double* partial;                 // [kProjQ][n_tiles * n_sub]
    double* coef;                    // [kProjMax n_inst]
    int32_t *kin, *kout;             // [n_inst] solutions available / basis size used
    int dw;                          // 1: double-word passes (D, Y and partial hold float pairs)
};
// hist: steps completed (device); lag: 1 when the initial field is not a solution (potential), 0 otherwise.
cudaError_t launch_projection(const ProjArgs& a, const int32_t* hist, int lag, cudaStream_t st);
// The same in two parts: the basis sizes and the basis (before the assembly when the assembly computes Y = A D),
// then [Y = A D if apply], the sums, the small solve and the guess with its residual.
cudaError_t launch_projection_basis(const ProjArgs& a, const int32_t* hist, int lag, cudaStream_t st);
cudaError_t launch_projection_rest(const ProjArgs& a, bool apply, cudaStream_t st);

// ---- monolithic step: flexible GMRES on the coupled Jacobian (mono_fgmres.cu) ---------------------------------
// Outer iterations of one Newton linear solve at most; the state lives in device memory so that every kernel of an
// outer iteration (and the inner persistent solves, through SolveArgs::skip) returns at once after convergence.
constexpr int kFgMax = 8;
struct FgState {
    int32_t done;                     // 1: converged, out of iterations, or broken down (the rest is skipped)
    int32_t k;                        // basis columns in the correction
    int32_t outer;                    // outer iterations taken
    int32_t status;                   // worst status of the inner solves (or RAFEM_ERR_NONFINITE)
    int32_t itV, itT;                 // inner Krylov iterations of the two systems
    int32_t single;                   // 1: the current column needed one Gram-Schmidt pass (the second is skipped)
    int32_t pad;
    double beta, eta, scale, ww;      // ||R||; forcing (relative); 1 / norm of the next basis vector; (w, w)
    double h[(kFgMax + 1) * kFgMax];  // Hessenberg, column j at h + j (kFgMax + 1), Givens-rotated
    double g[kFgMax + 1], cs[kFgMax], sn[kFgMax], y[kFgMax];
    double coef[kFgMax + 1];          // coefficients of the current Gram-Schmidt pass
};
// 2N-vector kernels of the solve: n2 = 2 N interleaved (V, T) entries; ld the stride of the basis arrays.
cudaError_t launch_fg_dots(int n2, const double* w, const double* V, size_t ld, int nv, const FgState* st,
                           double* partial, int G, cudaStream_t s, int pass = 1);
cudaError_t launch_fg_init(FgState* st, const double* partial, int G, double* newton_rr, double tol, cudaStream_t s);
cudaError_t launch_fg_scale(int n2, const double* src, double* dst, const FgState* st, cudaStream_t s);
cudaError_t launch_fg_split(int N, const double* v, double* rV, double* rT, double* zV, double* zT,
                            const FgState* st, cudaStream_t s);
cudaError_t launch_fg_count(FgState* st, const InstState* inst, int which, cudaStream_t s);
cudaError_t launch_fg_couple(int N, const int32_t* sp, const int32_t* sc, const int16_t* sc16, const double* vals4,
                             const double* zV, double* rT, const FgState* st, cudaStream_t s);
cudaError_t launch_fg_spmv(int N, const int32_t* sp, const int32_t* sc, const int16_t* sc16, const double* vals4,
                           const double* zV, const double* zT, double* w, double* Zj, const FgState* st,
                           cudaStream_t s);
cudaError_t launch_fg_gs(FgState* st, const double* partial, int G, int j, int pass, cudaStream_t s);
cudaError_t launch_fg_sub(int n2, double* w, const double* V, size_t ld, int j, const FgState* st, double* next,
                          int pass, cudaStream_t s);
cudaError_t launch_fg_finish(int n2, const double* Z, size_t ld, FgState* st, double* delta, InstState* instV,
                             InstState* instT, cudaStream_t s);
int fg_grid();

}  // namespace rafem
