// Persistent fused Krylov solvers: one cooperative launch runs a whole solve (all iterations) on the device.
//
// The paper solves each corrector pass's global system with library solvers (GMRES(m) to 1e-10 residual,
// Sec. III-B) and moves vector reductions to thrust (Sec. III-A). For the symmetric positive-definite lifted
// systems here, CG is the method of choice (Sec. II-B); it runs as one persistent kernel whose phases are
// separated by grid barriers, with every dot product fused into the phase that produces its operands:
//
//   Chronopoulos-Gear preconditioned CG (two grid barriers per iteration instead of three):
//     phase A (row-local):  p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,  u = M^-1 r,
//                           partial sums of gamma = (r, u) and rr = (r, r)
//     -- barrier --
//     phase B (SpMV):       w = A u,  partial sum of delta = (w, u)
//     -- barrier; the last block to arrive reduces the partial sums (fixed order: deterministic) and sets
//        beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev) per instance --
//
// Mixed precision (FP32 inner iterations, FP64 residual refinement): each instance runs a small state machine
// over the same rounds of [phase A, barrier, phase B, barrier + reduce]:
//     OUTER:   A: x64 += d32            B: r64 = b - A64 x64 (FP64 SpMV), r32 = (float) r64, d32 = 0,
//                                          u32 = M^-1 r32; sums rr64, gamma, rr32
//     START:   A: -                     B: w32 = A32 u32; sum delta
//     ITER:    A: FP32 CG vector update  B: w32 = A32 u32; sum delta
// FP64 appears only in the outer residual, the refinement update and the right-hand side.
//
// Work is split into tiles (contiguous row ranges, each belonging to one problem instance); blocks stride over
// tiles, and instances that have converged are skipped, so many independent systems of different sizes run
// in one launch (the batching form) with per-instance convergence.
//
// Storage: SELL-32 (slices of 32 rows, column-major, one thread per row) or CSR with 4..32 lanes per row.
// For SELL-32 the matrix stream is staged into shared memory by the Tensor Memory Accelerator: a producer
// warp issues bulk copies (cp.async.bulk, completion on mbarriers) of groups of slices into an 8-slot ring
// while 16 consumer warps compute on earlier groups, so the HBM stream keeps ~200 KB in flight per SM no
// matter how the consumers' gathers stall; the x gathers and the vector phases read L2, where the Krylov
// vectors stay because the matrix stream is loaded with an evict-first policy.
//
// Every grid barrier waits with a bounded spin (wall-clock limit); on expiry the kernel records
// RAFEM_ERR_TIMEOUT and returns instead of waiting forever.
#include <cuda_runtime.h>

#include <cmath>

#include "grid_sync.cuh"
#include "internal.h"
#include "sell_ring.cuh"

namespace rafem {

namespace {

using namespace sell;

enum { Q_GAMMA = 0, Q_RR = 1, Q_DELTA = 2, Q_BB = 3, Q_RR64 = 4, NQ_ALL = 5 };
static_assert(NQ_ALL == kPartialQ, "partial-sum buffer size");
enum { ST_OUTER = 1, ST_START = 2, ST_ITER = 3 };

// Grid barrier of the solver launch (bounded wait; see grid_sync.cuh). Returns true when the solve must stop
// because an error was recorded.
__device__ __forceinline__ bool grid_wait(const SolveArgs& a, unsigned& target) {
    return grid_barrier(a.bar, a.spin_limit_ns, target);
}

// SpMV over rows [r0, r1) of one tile in the context's storage: SELL-32 through the ring (L = 1: 32-bit columns,
// L = 2: 16-bit column deltas, L = 3: one column pattern per slice, values only) or CSR with L lanes per row.
template <int L, typename VT, typename AT, class Emit>
__device__ __forceinline__ bool spmv_tile(const SolveArgs& a, Ring& g, const VT* A, const VT* xin, int r0, int r1,
                                          const Emit& em) {
    if constexpr (L == 1) {
        return sell_tile<VT, AT>(a, g, a.rp, EntryCols<int32_t>{a.ci}, A, xin, r0, r1, em);
    } else if constexpr (L == 2) {
        return sell_tile<VT, AT>(a, g, a.rp, EntryCols<int16_t>{a.ci16}, A, xin, r0, r1, em);
    } else if constexpr (L == 3) {
        return sell_tile<VT, AT>(a, g, a.rp, SliceCols{a.pat_off, a.pat_pool, a.N}, A, xin, r0, r1, em);
    } else {
        csr_tile<L, VT, AT>(a.rp, a.ci, A, xin, r0, r1, em);
        return true;
    }
}

// ---- last-arriver reductions ---------------------------------------------------------------------------------

// After a barrier every block reduces the per-tile partial sums itself (fixed order: every block gets the same
// bits) and updates its own shared-memory copy of the per-instance solver state with fn(i, sums, state). Only
// active instances are visited. Returns the number of instances still active (block-uniform).
constexpr int kMaxInst = 96;

template <int NQ, class Fn>
__device__ __forceinline__ int reduce_shared(const SolveArgs& a, InstState* sst, Fn&& fn) {
    __shared__ double s_tot[NQ_ALL];
    __shared__ int s_active;
    if (a.n_inst == 1) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (sst[0].active && warp < NQ) {
            double acc = 0.0;
            for (int t = lane; t < a.n_tiles; t += 32) acc += ldcg(a.partial + (size_t)warp * a.n_tiles + t);
#pragma unroll
            for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) s_tot[warp] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sst[0].active) fn(0, s_tot, sst[0]);
            s_active = sst[0].active;
        }
        __syncthreads();
        return s_active;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < a.n_inst; i += kWarps) {
        if (!sst[i].active) continue;
        double v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = 0.0;
        const int t0 = a.inst_t0[i], t1 = a.inst_t1[i];
        for (int t = t0 + lane; t < t1; t += 32)
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[q] += ldcg(a.partial + (size_t)q * a.n_tiles + t);
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) fn(i, v, sst[i]);
    }
    if (threadIdx.x == 0) s_active = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < a.n_inst; i += kBlock) c += sst[i].active;
    if (c) atomicAdd(&s_active, c);
    __syncthreads();
    return s_active;
}

// Shared-memory solver state at kernel start: every instance active, first CG iteration pending.
__device__ __forceinline__ void init_shared_state(const SolveArgs& a, InstState* sst) {
    for (int i = threadIdx.x; i < a.n_inst; i += kBlock) {
        InstState z = {};
        z.active = 1;
        z.first = 1;
        z.outer = ST_OUTER;
        sst[i] = z;
    }
    __syncthreads();
}

// Block 0 publishes the final per-instance state (statistics) after the last barrier.
__device__ __forceinline__ void publish_state(const SolveArgs& a, const InstState* sst) {
    if (blockIdx.x != 0) return;
    for (int i = threadIdx.x; i < a.n_inst; i += kBlock) a.inst[i] = sst[i];
}

__device__ __forceinline__ void stop(InstState& st, int status) {
    st.status = status;
    st.active = 0;
}

// CG coefficients of the next iteration from gamma, delta; returns false (and stops) on breakdown.
__device__ __forceinline__ bool cg_coefficients(InstState& st, double gamma, double delta) {
    double alpha, beta;
    if (st.first) {
        beta = 0.0;
        if (!(delta > 0.0) || !(gamma > 0.0)) {
            stop(st, RAFEM_ERR_BREAKDOWN);
            return false;
        }
        alpha = gamma / delta;
    } else {
        beta = gamma / st.gamma_prev;
        const double den = delta - beta * gamma / st.alpha_prev;
        if (!(den > 0.0) || !(gamma > 0.0)) {
            stop(st, RAFEM_ERR_BREAKDOWN);
            return false;
        }
        alpha = gamma / den;
    }
    st.alpha = alpha;
    st.beta = beta;
    st.gamma_prev = gamma;
    st.alpha_prev = alpha;
    return true;
}

// FP32 coefficients of the inner iteration of the mixed solver (the inner solve runs in FP32 throughout).
__device__ __forceinline__ bool cg_coefficients32(InstState& st, float gamma, float delta) {
    const float beta = gamma / st.gprev32;
    const float den = delta - beta * gamma / st.aprev32;
    if (!(den > 0.0f) || !(gamma > 0.0f)) return false;
    const float alpha = gamma / den;
    st.alpha32 = alpha;
    st.beta32 = beta;
    st.gprev32 = gamma;
    st.aprev32 = alpha;
    return true;
}

// FP64 CG update of one instance at a reduce point.
__device__ __forceinline__ void cg_update(InstState& st, double gamma, double rr, double delta, double tol2,
                                          int max_iter, bool count_iter) {
    const double bb = st.bb > 0.0 ? st.bb : 1.0;
    if (count_iter) st.iters += 1;
    st.rr = rr;
    if (!isfinite(gamma) || !isfinite(rr) || !isfinite(delta)) return stop(st, RAFEM_ERR_NONFINITE);
    if (rr <= tol2 * bb) return stop(st, RAFEM_OK);
    if (st.iters >= max_iter) return stop(st, RAFEM_NOT_CONVERGED);
    cg_coefficients(st, gamma, delta);
}

// ---- phase helpers ------------------------------------------------------------------------------------------

// CG vector update of W consecutive rows (phase A) in type T; accumulates gamma and rr.
template <typename T, int W>
__device__ __forceinline__ void cg_vector_rows(int i, T alpha, T beta, bool first, T* x, T* r, T* u, const T* w,
                                               T* p, T* s, const T* dinv, T& g, T& rr) {
    Vec<T, W> ui = ldv<T, W>(u + i), wi = ldv<T, W>(w + i), xi = ldv<T, W>(x + i), ri = ldv<T, W>(r + i),
              di = ldv<T, W>(dinv + i);
    Vec<T, W> pi, si;
    if (first) {
        pi = ui;
        si = wi;
    } else {
        pi = ldv<T, W>(p + i);
        si = ldv<T, W>(s + i);
#pragma unroll
        for (int k = 0; k < W; ++k) {
            pi.v[k] = fma(beta, pi.v[k], ui.v[k]);
            si.v[k] = fma(beta, si.v[k], wi.v[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
        xi.v[k] = fma(alpha, pi.v[k], xi.v[k]);
        ri.v[k] = fma(-alpha, si.v[k], ri.v[k]);
        ui.v[k] = di.v[k] * ri.v[k];
        g = fma(ri.v[k], ui.v[k], g);
        rr = fma(ri.v[k], ri.v[k], rr);
    }
    stv<T, W>(p + i, pi);
    stv<T, W>(s + i, si);
    stv<T, W>(x + i, xi);
    stv<T, W>(r + i, ri);
    stv<T, W>(u + i, ui);
}

template <typename T, int W>
struct CgLoad {
    Vec<T, W> u, w, x, r, d, p, s;
};
template <typename T, int W>
__device__ __forceinline__ CgLoad<T, W> cg_load(int i, bool first, const T* x, const T* r, const T* u, const T* w,
                                               const T* p, const T* s, const T* dinv) {
    CgLoad<T, W> L;
    L.u = ldv<T, W>(u + i);
    L.w = ldv<T, W>(w + i);
    L.x = ldv<T, W>(x + i);
    L.r = ldv<T, W>(r + i);
    L.d = ldv<T, W>(dinv + i);
    if (!first) {
        L.p = ldv<T, W>(p + i);
        L.s = ldv<T, W>(s + i);
    }
    return L;
}
template <typename T, int W>
__device__ __forceinline__ void cg_apply(int i, CgLoad<T, W>& L, T alpha, T beta, bool first, T* x, T* r, T* u, T* p,
                                         T* s, T& g, T& rr) {
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const T pi = first ? L.u.v[k] : fma(beta, L.p.v[k], L.u.v[k]);
        const T si = first ? L.w.v[k] : fma(beta, L.s.v[k], L.w.v[k]);
        L.p.v[k] = pi;
        L.s.v[k] = si;
        L.x.v[k] = fma(alpha, pi, L.x.v[k]);
        const T ri = fma(-alpha, si, L.r.v[k]);
        L.r.v[k] = ri;
        const T ui = L.d.v[k] * ri;
        L.u.v[k] = ui;
        g = fma(ri, ui, g);
        rr = fma(ri, ri, rr);
    }
    stv<T, W>(p + i, L.p);
    stv<T, W>(s + i, L.s);
    stv<T, W>(x + i, L.x);
    stv<T, W>(r + i, L.r);
    stv<T, W>(u + i, L.u);
}
template <typename T, int W>
__device__ __forceinline__ void cg_vector_rows2(int i, int j, T alpha, T beta, bool first, T* x, T* r, T* u,
                                                const T* w, T* p, T* s, const T* dinv, T& g, T& rr) {
    CgLoad<T, W> A = cg_load<T, W>(i, first, x, r, u, w, p, s, dinv);
    CgLoad<T, W> B = cg_load<T, W>(j, first, x, r, u, w, p, s, dinv);
    cg_apply<T, W>(i, A, alpha, beta, first, x, r, u, p, s, g, rr);
    cg_apply<T, W>(j, B, alpha, beta, first, x, r, u, p, s, g, rr);
}

template <typename T>
struct CgRows {
    T* x;
    T* r;
    T* u;
    const T* w;
    T* p;
    T* s;
    const T* dinv;
    T alpha, beta;
    bool first;
    T* v;
    template <int W>
    __device__ __forceinline__ void operator()(int i) const {
        cg_vector_rows<T, W>(i, alpha, beta, first, x, r, u, w, p, s, dinv, v[0], v[1]);
    }
    // two independent groups: every load of both is issued before the first store
    template <int W>
    __device__ __forceinline__ void pair(int i, int j) const {
        cg_vector_rows2<T, W>(i, j, alpha, beta, first, x, r, u, w, p, s, dinv, v[0], v[1]);
    }
};

// ---- emitters (row-local work fused into the SpMV) ----------------------------------------------------------

// r = b - A x, dinv = 1 / a_ii, partial bb += b^2
struct EmInitResidual {
    const SolveArgs& a;
    double* v;
    __device__ __forceinline__ double pre(int row) const { return a.b[row]; }
    __device__ __forceinline__ void fin(int row, double ax, double bi) const { fin_res(row, bi - ax, bi); }
    // the residual given (see given_residual)
    __device__ __forceinline__ void fin_res(int row, double r, double bi) const {
        a.r[row] = r;
        a.dinv[row] = 1.0 / a.A[a.diag[row]];
        v[0] = fma(bi, bi, v[0]);
    }
};

// Whether the starting residual b - A x of tile t's instance was computed by the predictor (SolveArgs::r0), so
// that the first residual pass reads it instead of running an SpMV (block-uniform).
__device__ __forceinline__ bool given_residual(const SolveArgs& a, int t) {
    return a.r0 != nullptr && a.r0_ok[a.tile_inst[t]] > 0;
}
template <class Emit>
__device__ __forceinline__ void given_residual_rows(const SolveArgs& a, int r0, int r1, const Emit& em) {
    for (int row = r0 + threadIdx.x; row < r1; row += kBlock) em.fin_res(row, ldcg(a.r0 + row), em.pre(row));
}

// w = A u, partial delta += w u
template <typename T>
struct EmAu {
    T* w;
    const T* u;
    T* v;
    __device__ __forceinline__ T pre(int row) const { return ldcg(u + row); }
    __device__ __forceinline__ void fin(int row, T wu, T ui) const {
        w[row] = wu;
        v[0] = fma(wu, ui, v[0]);
    }
};

// partial ||b - A x||^2
struct EmTrueResidual {
    const double* b;
    double* v;
    __device__ __forceinline__ double pre(int row) const { return b[row]; }
    __device__ __forceinline__ void fin(int, double ax, double bi) const {
        const double r = bi - ax;
        v[0] = fma(r, r, v[0]);
    }
};

// ---- FP64 Chronopoulos-Gear Jacobi-PCG ----------------------------------------------------------------------

template <int L>
__global__ void __launch_bounds__(kBlock, 1) k_cg64(SolveArgs a) {
    if (a.skip && *(volatile const int*)a.skip) return;  // an outer iteration that is not needed
    RAFEM_RING_SETUP(L)
    __shared__ double sm[kSumMax * kBlock];
    __shared__ InstState sst[kMaxInst];
    init_shared_state(a, sst);
    const int nt = a.n_tiles;
    const double tol2 = a.tol * a.tol;
    unsigned target = 0;
    bool ok = true;

    // init 1: r = b - A x (or the predictor's residual), dinv, bb
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
        double v[1] = {0.0};
        if (given_residual(a, t))
            given_residual_rows(a, r0, r1, EmInitResidual{a, v});
        else
            ok = spmv_tile<L, double, double>(a, ring, a.A, a.x, r0, r1, EmInitResidual{a, v}) && ok;
        block_sum<1>(v, sm);
        if (threadIdx.x == 0) a.partial[(size_t)Q_BB * nt + t] = v[0];
    }
    __syncthreads();
    // init 2 only needs row-local data of init 1 (same tiles, same block): u = dinv r; gamma, rr
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
        double v[2] = {0.0, 0.0};
        for (int i = r0 + threadIdx.x; i < r1; i += kBlock) {
            const double ri = ldcg(a.r + i);
            const double ui = ldcg(a.dinv + i) * ri;
            a.u[i] = ui;
            v[0] += ri * ui;
            v[1] += ri * ri;
        }
        block_sum<2>(v, sm);
        if (threadIdx.x == 0) {
            a.partial[(size_t)Q_GAMMA * nt + t] = v[0];
            a.partial[(size_t)Q_RR * nt + t] = v[1];
        }
    }
    if (grid_wait(a, target) || !ok) return;
    // init 3: w = A u; delta
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
        double v[1] = {0.0};
        ok = spmv_tile<L, double, double>(a, ring, a.A, a.u, r0, r1, EmAu<double>{a.w, a.u, v}) && ok;
        block_sum<1>(v, sm);
        if (threadIdx.x == 0) a.partial[(size_t)Q_DELTA * nt + t] = v[0];
    }
    if (grid_wait(a, target) || !ok) return;
    int n_active = reduce_shared<4>(a, sst, [&](int, const double* s, InstState& st) {
        st.bb = s[Q_BB];
        st.first = 1;
        cg_update(st, s[Q_GAMMA], s[Q_RR], s[Q_DELTA], tol2, a.max_iter, false);
    });

    while (n_active > 0) {
        // phase A
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState& st = sst[a.tile_inst[t]];
            if (!st.active) continue;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[2] = {0.0, 0.0};
            CgRows<double> f{a.x, a.r, a.u, a.w, a.p, a.s, a.dinv, st.alpha, st.beta, st.first != 0, v};
            for_rows<2>(r0, r1, f);
            block_sum<2>(v, sm);
            if (threadIdx.x == 0) {
                a.partial[(size_t)Q_GAMMA * nt + t] = v[0];
                a.partial[(size_t)Q_RR * nt + t] = v[1];
            }
        }
        if (grid_wait(a, target)) return;
        // phase B
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState& st = sst[a.tile_inst[t]];
            if (!st.active) continue;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[1] = {0.0};
            ok = spmv_tile<L, double, double>(a, ring, a.A, a.u, r0, r1, EmAu<double>{a.w, a.u, v}) && ok;
            block_sum<1>(v, sm);
            if (threadIdx.x == 0) a.partial[(size_t)Q_DELTA * nt + t] = v[0];
        }
        if (grid_wait(a, target) || !ok) return;
        n_active = reduce_shared<3>(a, sst, [&](int, const double* s, InstState& st) {
            st.first = 0;
            cg_update(st, s[Q_GAMMA], s[Q_RR], s[Q_DELTA], tol2, a.max_iter, true);
        });
    }

    // final: true residual ||b - A x|| for the reported relative residual
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
        double v[1] = {0.0};
        ok = spmv_tile<L, double, double>(a, ring, a.A, a.x, r0, r1, EmTrueResidual{a.b, v}) && ok;
        block_sum<1>(v, sm);
        if (threadIdx.x == 0) a.partial[(size_t)Q_RR * nt + t] = v[0];
    }
    if (grid_wait(a, target) || !ok) return;
    if (blockIdx.x == 0) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int i = warp; i < a.n_inst; i += kWarps) {
            double v = 0.0;
            for (int t = a.inst_t0[i] + lane; t < a.inst_t1[i]; t += 32) v += ldcg(a.partial + (size_t)Q_RR * nt + t);
#pragma unroll
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                InstState& st = sst[i];
                const double bb = st.bb > 0.0 ? st.bb : 1.0;
                st.relres = sqrt(v / bb);
                if (!isfinite(v) && st.status >= 0) st.status = RAFEM_ERR_NONFINITE;
            }
        }
        __syncthreads();
        publish_state(a, sst);
    }
}

// ---- FP64 pipelined Jacobi-PCG ---------------------------------------------------------------------------------
// Ghysels and Vanroose, "Hiding global synchronization latency in the preconditioned Conjugate Gradient
// algorithm", Parallel Computing 40(7), 2014: the same iterates as CG in exact arithmetic, with the dot products
// of an iteration computed from vectors that already exist when its SpMV starts. In this persistent kernel that
// leaves ONE grid barrier per iteration: after it every block reduces (gamma_i, delta_i, rr_i), forms alpha_i and
// beta_i, and runs n_i = A m_i with every vector update fused into the rows' epilogue:
//   z = n + beta z,  q = m + beta q,  s = w + beta s,  p = u + beta p,
//   x += alpha p,  r -= alpha s,  u -= alpha q,  w -= alpha z,  m' = M^-1 w,
//   partial sums gamma' = (r, u), delta' = (w, u), rr' = (r, r)
// (n is never stored). m is double-buffered: the SpMV of iteration i gathers m_i from other tiles while rows
// write m_{i+1}. The recurrences drift further from the true residual than CG's, so a solve ends with the true
// residual and restarts from the current x (residual replacement) while it misses the target, at most
// kPipeRestarts times. It trades one barrier per iteration for 20 vector touches instead of 14: a gain where
// barriers dominate (small systems, batches of small instances), a loss where the vector streams do.
constexpr int kPipeRestarts = 3;

// w = A u at start-up; m = M^-1 w, partials gamma = (r, u), delta = (w, u), rr = (r, r)
struct EmPipeInit {
    const SolveArgs& a;
    double* m;
    double* v;
    __device__ __forceinline__ double pre(int row) const { return ldcg(a.u + row); }
    __device__ __forceinline__ void fin(int row, double wi, double ui) const {
        const double ri = ldcg(a.r + row);
        a.w[row] = wi;
        m[row] = ldcg(a.dinv + row) * wi;
        v[0] = fma(ri, ui, v[0]);
        v[1] = fma(wi, ui, v[1]);
        v[2] = fma(ri, ri, v[2]);
    }
};

// one pipelined iteration's row epilogue (see above); n = (A m_in)_row
struct EmPipe {
    const SolveArgs& a;
    const double* m_in;
    double* m_out;
    double alpha, beta;
    bool first;
    double* v;
    __device__ __forceinline__ double pre(int row) const { return ldcg(m_in + row); }
    __device__ __forceinline__ void fin(int row, double n, double mi) const {
        const double wi = ldcg(a.w + row), ui = ldcg(a.u + row);
        double zi, qi, si, pi;
        if (first) {
            zi = n;
            qi = mi;
            si = wi;
            pi = ui;
        } else {
            zi = fma(beta, ldcg(a.z + row), n);
            qi = fma(beta, ldcg(a.q + row), mi);
            si = fma(beta, ldcg(a.s + row), wi);
            pi = fma(beta, ldcg(a.p + row), ui);
        }
        const double xi = fma(alpha, pi, ldcg(a.x + row));
        const double ri = fma(-alpha, si, ldcg(a.r + row));
        const double un = fma(-alpha, qi, ui);
        const double wn = fma(-alpha, zi, wi);
        a.z[row] = zi;
        a.q[row] = qi;
        a.s[row] = si;
        a.p[row] = pi;
        a.x[row] = xi;
        a.r[row] = ri;
        a.u[row] = un;
        a.w[row] = wn;
        m_out[row] = ldcg(a.dinv + row) * wn;
        v[0] = fma(ri, un, v[0]);
        v[1] = fma(wn, un, v[1]);
        v[2] = fma(ri, ri, v[2]);
    }
};

template <int L>
__global__ void __launch_bounds__(kBlock, 1) k_pcg64(SolveArgs a) {
    if (a.skip && *(volatile const int*)a.skip) return;  // an outer iteration that is not needed
    RAFEM_RING_SETUP(L)
    __shared__ double sm[kSumMax * kBlock];
    __shared__ InstState sst[kMaxInst];
    init_shared_state(a, sst);
    const int nt = a.n_tiles;
    const double tol2 = a.tol * a.tol;
    unsigned target = 0;
    bool ok = true;
    int n_active = a.n_inst;
    for (int restart = 0; n_active > 0; ++restart) {
        // init 1: r = b - A x, dinv, bb; u = dinv r (row-local, same block)
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            if (!sst[a.tile_inst[t]].active) continue;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[1] = {0.0};
            ok = spmv_tile<L, double, double>(a, ring, a.A, a.x, r0, r1, EmInitResidual{a, v}) && ok;
            block_sum<1>(v, sm);
            if (threadIdx.x == 0) a.partial[(size_t)Q_BB * nt + t] = v[0];
            for (int i = r0 + threadIdx.x; i < r1; i += kBlock) a.u[i] = ldcg(a.dinv + i) * ldcg(a.r + i);
        }
        if (grid_wait(a, target) || !ok) return;
        // init 2: w = A u, m_0, gamma, delta, rr
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            if (!sst[a.tile_inst[t]].active) continue;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[3] = {0.0, 0.0, 0.0};
            ok = spmv_tile<L, double, double>(a, ring, a.A, a.u, r0, r1, EmPipeInit{a, a.ma, v}) && ok;
            double v2[2] = {v[0], v[1]}, v1[1] = {v[2]};
            block_sum<2>(v2, sm);
            block_sum<1>(v1, sm);
            if (threadIdx.x == 0) {
                a.partial[(size_t)Q_GAMMA * nt + t] = v2[0];
                a.partial[(size_t)Q_DELTA * nt + t] = v2[1];
                a.partial[(size_t)Q_RR * nt + t] = v1[0];
            }
        }
        if (grid_wait(a, target) || !ok) return;
        n_active = reduce_shared<4>(a, sst, [&](int, const double* s, InstState& st) {
            st.bb = s[Q_BB];
            st.first = 1;
            cg_update(st, s[Q_GAMMA], s[Q_RR], s[Q_DELTA], tol2, a.max_iter, false);
        });
        int parity = 0;
        while (n_active > 0) {
            const double* m_in = parity ? a.mb : a.ma;
            double* m_out = parity ? a.ma : a.mb;
            for (int t = blockIdx.x; t < nt; t += gridDim.x) {
                const InstState& st = sst[a.tile_inst[t]];
                if (!st.active) continue;
                const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
                double v[3] = {0.0, 0.0, 0.0};
                ok = spmv_tile<L, double, double>(
                         a, ring, a.A, m_in, r0, r1,
                         EmPipe{a, m_in, m_out, st.alpha, st.beta, st.first != 0, v}) &&
                     ok;
                double v2[2] = {v[0], v[1]}, v1[1] = {v[2]};
                block_sum<2>(v2, sm);
                block_sum<1>(v1, sm);
                if (threadIdx.x == 0) {
                    a.partial[(size_t)Q_GAMMA * nt + t] = v2[0];
                    a.partial[(size_t)Q_DELTA * nt + t] = v2[1];
                    a.partial[(size_t)Q_RR * nt + t] = v1[0];
                }
            }
            parity ^= 1;
            if (grid_wait(a, target) || !ok) return;
            n_active = reduce_shared<3>(a, sst, [&](int, const double* s, InstState& st) {
                st.first = 0;
                cg_update(st, s[Q_GAMMA], s[Q_RR], s[Q_DELTA], tol2, a.max_iter, true);
            });
        }
        // true residual ||b - A x|| of every instance; those that converged by their recurrence but miss the
        // target start again from x (residual replacement)
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[1] = {0.0};
            ok = spmv_tile<L, double, double>(a, ring, a.A, a.x, r0, r1, EmTrueResidual{a.b, v}) && ok;
            block_sum<1>(v, sm);
            if (threadIdx.x == 0) a.partial[(size_t)Q_RR64 * nt + t] = v[0];
        }
        if (grid_wait(a, target) || !ok) return;
        {
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            __shared__ int s_restart;
            if (threadIdx.x == 0) s_restart = 0;
            __syncthreads();
            for (int i = warp; i < a.n_inst; i += kWarps) {
                double v = 0.0;
                for (int t = a.inst_t0[i] + lane; t < a.inst_t1[i]; t += 32)
                    v += ldcg(a.partial + (size_t)Q_RR64 * nt + t);
#pragma unroll
                for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) {
                    InstState& st = sst[i];
                    const double bb = st.bb > 0.0 ? st.bb : 1.0;
                    st.relres = sqrt(v / bb);
                    if (!isfinite(v)) {
                        if (st.status >= 0) st.status = RAFEM_ERR_NONFINITE;
                    } else if (st.status == RAFEM_OK && v > tol2 * bb) {
                        if (restart < kPipeRestarts && st.iters < a.max_iter) {
                            st.active = 1;
                            st.status = 0;
                            atomicAdd(&s_restart, 1);
                        } else {
                            st.status = RAFEM_NOT_CONVERGED;
                        }
                    }
                }
            }
            __syncthreads();
            n_active = s_restart;
            __syncthreads();
        }
    }
    publish_state(a, sst);
}

// ---- mixed precision: FP32 Chronopoulos-Gear inner iterations, FP64 residual refinement ---------------------
// Each instance runs a state machine over rounds of [phase A, barrier, phase B, barrier + reduce]:
//   OUTER: A: x64 += d32 (after an inner solve)   B: r64 = b - A64 x64 (FP64 SpMV), r32 = (float) r64, d32 = 0,
//                                                    u32 = M^-1 r32; sums bb, rr64, gamma, rr32
//   START: A: -                                   B: w32 = A32 u32; sum delta
//   ITER:  A: FP32 CG vector update                B: w32 = A32 u32; sum delta
// An inner solve ends at inner_tol, at the predicted outer target, or when its FP32 recurrence loses positive
// curvature; the FP64 residual then starts the next one.

struct EmOuter {
    const SolveArgs& a;
    double* v;  // [bb, rr64]
    float* f;   // [gamma, rr32]
    struct P {
        double b;
        float dinv;
    };
    __device__ __forceinline__ P pre(int row) const { return P{a.b[row], ldcg(a.dinv32 + row)}; }
    __device__ __forceinline__ void fin(int row, double ax, const P& p) const { fin_res(row, p.b - ax, p); }
    __device__ __forceinline__ void fin_res(int row, double r64, const P& p) const {
        const float r32 = (float)r64;
        const float u32 = p.dinv * r32;
        a.r32[row] = r32;
        a.u32[row] = u32;
        a.d32[row] = 0.0f;
        v[0] = fma(p.b, p.b, v[0]);
        v[1] = fma(r64, r64, v[1]);
        f[0] = fmaf(r32, u32, f[0]);
        f[1] = fmaf(r32, r32, f[1]);
    }
};

// x64 += (double) d32 over W consecutive rows (W = 1 or 4).
struct AddCorrection {
    double* x;
    const float* d;
    template <int W>
    __device__ __forceinline__ void pair(int i, int j) const {
        operator()<W>(i);
        operator()<W>(j);
    }
    template <int W>
    __device__ __forceinline__ void operator()(int i) const {
        if constexpr (W == 1) {
            x[i] = ldcg(x + i) + (double)ldcg(d + i);
        } else {
            Vec<double, 2> x0 = ldv<double, 2>(x + i), x1 = ldv<double, 2>(x + i + 2);
            Vec<float, 4> di = ldv<float, 4>(d + i);
            x0.v[0] += (double)di.v[0];
            x0.v[1] += (double)di.v[1];
            x1.v[0] += (double)di.v[2];
            x1.v[1] += (double)di.v[3];
            stv<double, 2>(x + i, x0);
            stv<double, 2>(x + i + 2, x1);
        }
    }
};

template <int L>
__global__ void __launch_bounds__(kBlock, 1) k_cg_mixed(SolveArgs a) {
    if (a.skip && *(volatile const int*)a.skip) return;  // an outer iteration that is not needed
    RAFEM_RING_SETUP(L)
    __shared__ double sm[kSumMax * kBlock];
    __shared__ InstState sst[kMaxInst];
    init_shared_state(a, sst);
    const int nt = a.n_tiles;
    const double tol2 = a.tol * a.tol;
    const double itol2 = a.inner_tol * a.inner_tol;
    unsigned target = 0;
    bool ok = true;

    // init: dinv32 from the FP32 diagonal (row-local; read again only by the same block after a barrier). The
    // rows of a thread are taken eight at a time so that their slot and diagonal loads overlap.
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r1 = a.tile_r1[t];
        for (int i0 = a.tile_r0[t] + threadIdx.x; i0 < r1; i0 += 8 * kBlock) {
            int slot[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) slot[k] = i0 + k * kBlock < r1 ? __ldg(a.diag + i0 + k * kBlock) : -1;
            float dv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) dv[k] = slot[k] >= 0 ? __ldcg(a.A32 + slot[k]) : 1.0f;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (slot[k] >= 0) a.dinv32[i0 + k * kBlock] = 1.0f / dv[k];
        }
    }
    __syncthreads();
    bool first_round = true;
    int n_active = a.n_inst;
    while (n_active > 0) {
        // ---------------- phase A ----------------
        if (!first_round) {
            for (int t = blockIdx.x; t < nt; t += gridDim.x) {
                const InstState& st = sst[a.tile_inst[t]];
                if (!st.active) continue;
                const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
                if (st.outer == ST_OUTER) {
                    for_rows<4>(r0, r1, AddCorrection{a.x, a.d32});
                } else if (st.outer == ST_ITER) {
                    float v[2] = {0.0f, 0.0f};
                    CgRows<float> f{a.d32, a.r32, a.u32, a.w32, a.p32, a.s32, a.dinv32, st.alpha32, st.beta32,
                                    st.first != 0, v};
                    for_rows<4>(r0, r1, f);
                    double vd[2] = {(double)v[0], (double)v[1]};
                    block_sum<2>(vd, sm);
                    if (threadIdx.x == 0) {
                        a.partial[(size_t)Q_GAMMA * nt + t] = vd[0];
                        a.partial[(size_t)Q_RR * nt + t] = vd[1];
                    }
                }
            }
            if (grid_wait(a, target)) return;
        }
        // ---------------- phase B ----------------
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState& st = sst[a.tile_inst[t]];
            if (!st.active) continue;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            if (st.outer == ST_OUTER) {
                double v[2] = {0.0, 0.0};
                float f[2] = {0.0f, 0.0f};
                // the first residual of the solve may come from the predictor (no SpMV)
                if (first_round && given_residual(a, t))
                    given_residual_rows(a, r0, r1, EmOuter{a, v, f});
                else
                    ok = spmv_tile<L, double, double>(a, ring, a.A, a.x, r0, r1, EmOuter{a, v, f}) && ok;
                block_sum<2>(v, sm);
                double fd[2] = {(double)f[0], (double)f[1]};
                block_sum<2>(fd, sm);
                if (threadIdx.x == 0) {
                    a.partial[(size_t)Q_BB * nt + t] = v[0];
                    a.partial[(size_t)Q_RR64 * nt + t] = v[1];
                    a.partial[(size_t)Q_GAMMA * nt + t] = fd[0];
                    a.partial[(size_t)Q_RR * nt + t] = fd[1];
                }
            } else {
                float v[1] = {0.0f};
                ok = spmv_tile<L, float, float>(a, ring, a.A32, a.u32, r0, r1, EmAu<float>{a.w32, a.u32, v}) && ok;
                double vd[1] = {(double)v[0]};
                block_sum<1>(vd, sm);
                if (threadIdx.x == 0) a.partial[(size_t)Q_DELTA * nt + t] = vd[0];
            }
        }
        first_round = false;
        if (grid_wait(a, target) || !ok) return;
        n_active = reduce_shared<NQ_ALL>(a, sst, [&](int, const double* s, InstState& st) {
            if (st.outer == ST_OUTER) {
                // FP64 residual of the current x: converged, capped, or start an inner solve
                st.bb = s[Q_BB];
                const double bb = st.bb > 0.0 ? st.bb : 1.0;
                const double rr64 = s[Q_RR64];
                st.relres = sqrt(rr64 / bb);
                st.rr0 = rr64;
                if (!isfinite(rr64)) {
                    stop(st, RAFEM_ERR_NONFINITE);
                } else if (rr64 <= tol2 * bb) {
                    stop(st, RAFEM_OK);
                } else if (st.refine >= a.max_refine || st.iters >= a.max_iter) {
                    stop(st, RAFEM_NOT_CONVERGED);
                } else {
                    st.refine += 1;
                    st.outer = ST_START;
                    st.gamma = s[Q_GAMMA];
                    st.rr_in0 = s[Q_RR];
                    st.first = 1;
                }
            } else if (st.outer == ST_START) {
                st.first = 1;
                const float gamma = (float)st.gamma, delta = (float)s[Q_DELTA];
                if (!isfinite(s[Q_DELTA])) {
                    stop(st, RAFEM_ERR_NONFINITE);
                } else if (!(delta > 0.0f) || !(gamma > 0.0f)) {
                    stop(st, RAFEM_ERR_BREAKDOWN);
                } else {
                    st.alpha32 = gamma / delta;
                    st.beta32 = 0.0f;
                    st.gprev32 = gamma;
                    st.aprev32 = st.alpha32;
                    // the inner solve stops at inner_tol, or once the predicted outer residual
                    // ||r64|| * ||r32|| / ||r32_0|| reaches the outer tolerance (a stricter margin only adds
                    // FP32 iterations: the next FP64 residual decides convergence either way)
                    const double bb = st.bb > 0.0 ? st.bb : 1.0;
                    st.thr32 = (float)(fmax(itol2, tol2 * bb / fmax(st.rr0, 1e-300)) * st.rr_in0);
                    st.outer = ST_ITER;
                }
            } else {
                // ST_ITER: one inner FP32 iteration done
                st.iters += 1;
                st.first = 0;
                const float rr = (float)s[Q_RR], gamma = (float)s[Q_GAMMA], delta = (float)s[Q_DELTA];
                if (!isfinite(rr) || !isfinite(gamma) || !isfinite(delta)) {
                    stop(st, RAFEM_ERR_NONFINITE);
                } else if (rr <= st.thr32 || st.iters >= a.max_iter) {
                    st.outer = ST_OUTER;
                } else if (!cg_coefficients32(st, gamma, delta)) {
                    // FP32 recurrence lost positive curvature: keep the correction found so far and let
                    // the FP64 residual start the next inner solve
                    st.outer = ST_OUTER;
                    st.breakdowns += 1;
                }
            }
        });
    }
    publish_state(a, sst);
}

__global__ void k_reset(InstState* inst, int n_inst, GridBarrier* bar, int missing) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
        InstState z = {};
        z.active = 1;
        z.first = 1;
        z.outer = ST_OUTER;
        inst[i] = z;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bar->count = 0u - (unsigned)missing;
        bar->err = 0;
        bar->n_active = n_inst;
    }
}

__global__ void k_barrier_reset(GridBarrier* bar, int missing) {
    bar->count = 0u - (unsigned)missing;
    bar->err = 0;
}

template <int L>
void* kernel_ptr(int precision, bool pipelined) {
    if (pipelined) return precision == RAFEM_PRECISION_FP64 ? (void*)k_pcg64<L> : nullptr;
    return precision == RAFEM_PRECISION_MIXED ? (void*)k_cg_mixed<L> : (void*)k_cg64<L>;
}

void* select_kernel(int lanes, int precision, bool pipelined) {
    switch (lanes) {
        case 1: return kernel_ptr<1>(precision, pipelined);
        case 2: return kernel_ptr<2>(precision, pipelined);
        case 3: return kernel_ptr<3>(precision, pipelined);
        case 4: return kernel_ptr<4>(precision, pipelined);
        case 8: return kernel_ptr<8>(precision, pipelined);
        case 16: return kernel_ptr<16>(precision, pipelined);
        case 32: return kernel_ptr<32>(precision, pipelined);
        default: return nullptr;
    }
}

}  // namespace

cudaError_t launch_barrier_reset(GridBarrier* bar, int missing, cudaStream_t st) {
    k_barrier_reset<<<1, 1, 0, st>>>(bar, missing);
    return cudaGetLastError();
}

// Dynamic shared memory of a solver launch: the bulk-copy ring for SELL-32 (codes 1-3), none for CSR.
static int dyn_smem(int lanes) { return lanes <= 3 ? kRingBytes : 0; }

int krylov_max_blocks(int lanes, int precision, bool pipelined, int* block_threads) {
    void* k = select_kernel(lanes, precision, pipelined);
    if (!k) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem(lanes)) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlock, dyn_smem(lanes)) != cudaSuccess) return 0;
    if (block_threads) *block_threads = kBlock;
    return per_sm * sms;
}

cudaError_t launch_krylov(const SolveArgs& a, int lanes, int precision, bool pipelined, int grid, int block,
                          cudaStream_t st) {
    void* k = select_kernel(lanes, precision, pipelined);
    if (!k) return cudaErrorInvalidValue;
    k_reset<<<(a.n_inst + 255) / 256, 256, 0, st>>>(a.inst, a.n_inst, a.bar, a.bar_missing);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = dyn_smem(lanes);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SolveArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace rafem
