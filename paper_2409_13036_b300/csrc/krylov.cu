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
// Storage: SELL-32 (slices of 32 rows, column-major, one thread per row: coalesced loads, every entry of a row
// an independent load) or CSR with 4..32 lanes per row.
//
// Every grid barrier waits with a bounded spin (wall-clock limit); on expiry the kernel records
// RAFEM_ERR_TIMEOUT and returns instead of waiting forever.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace rafem {

namespace {

constexpr int kBlock = 256;
constexpr int kWarps = kBlock / 32;

enum { Q_GAMMA = 0, Q_RR = 1, Q_DELTA = 2, Q_BB = 3, Q_RR64 = 4, NQ_ALL = 5 };
enum { ST_OUTER = 1, ST_START = 2, ST_ITER = 3 };

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Loads of data written by other blocks during the kernel go through L2 (L1 is not coherent).
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ int ldcg(const int* p) { return __ldcg(p); }

// W consecutive values loaded/stored as one vector access (W = 1, 2 for double; 1, 4 for float).
template <typename T, int W>
struct Vec {
    T v[W];
};
template <typename T, int W>
__device__ __forceinline__ Vec<T, W> ldv(const T* p) {
    Vec<T, W> r;
    if constexpr (W == 1) {
        r.v[0] = __ldcg(p);
    } else if constexpr (sizeof(T) == 8 && W == 2) {
        double2 q = __ldcg(reinterpret_cast<const double2*>(p));
        r.v[0] = q.x;
        r.v[1] = q.y;
    } else {
        static_assert(sizeof(T) == 4 && W == 4, "vector width");
        float4 q = __ldcg(reinterpret_cast<const float4*>(p));
        r.v[0] = q.x;
        r.v[1] = q.y;
        r.v[2] = q.z;
        r.v[3] = q.w;
    }
    return r;
}
template <typename T, int W>
__device__ __forceinline__ void stv(T* p, const Vec<T, W>& r) {
    if constexpr (W == 1) {
        p[0] = r.v[0];
    } else if constexpr (sizeof(T) == 8 && W == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
    } else {
        *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    }
}

// Visit rows [r0, r1) of a tile: aligned groups of W rows as f.template operator()<W>(i), the unaligned head
// and tail one row at a time.
template <int W, class F>
__device__ __forceinline__ void for_rows(int r0, int r1, const F& f) {
    int a0 = (r0 + W - 1) / W * W;
    if (a0 > r1) a0 = r1;
    const int a1 = a0 + (r1 - a0) / W * W;
    for (int i = r0 + threadIdx.x; i < a0; i += kBlock) f.template operator()<1>(i);
    for (int i = a0 + W * threadIdx.x; i < a1; i += W * kBlock) f.template operator()<W>(i);
    for (int i = a1 + threadIdx.x; i < r1; i += kBlock) f.template operator()<1>(i);
}

// Block-wide sum of NQ values with a fixed reduction tree; result valid in thread 0.
template <int NQ, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NQ], T* sm /* [NQ*32] */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) sm[q * 32 + warp] = v[q];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            v[q] = lane < kWarps ? sm[q * 32 + lane] : T(0);
#pragma unroll
            for (int o = 16; o; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        }
    }
    __syncthreads();
}

// Grid barrier. The last block to arrive runs `last` (whole block) before releasing the others.
// Returns true when the solve must stop because an error was recorded.
template <class F>
__device__ __forceinline__ bool grid_sync(const SolveArgs& a, F&& last) {
    __shared__ unsigned s_gen;
    __shared__ int s_last, s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g = ld_acquire_u32(&a.bar->gen);
        __threadfence();
        unsigned t = atomicAdd(&a.bar->count, 1u);
        s_gen = g;
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        last();
        __syncthreads();
        if (threadIdx.x == 0) {
            a.bar->count = 0;
            __threadfence();
            st_release_u32(&a.bar->gen, s_gen + 1);
        }
    } else if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        long long spins = 0;
        while (ld_acquire_u32(&a.bar->gen) == s_gen) {
            ++spins;
            if ((spins & 255) == 0 &&
                ((long long)(globaltimer() - t0) > a.spin_limit_ns || spins > (1LL << 40))) {
                atomicExch(&a.bar->err, RAFEM_ERR_TIMEOUT);
                break;
            }
        }
    }
    if (threadIdx.x == 0) s_err = *(volatile int*)&a.bar->err;
    __syncthreads();
    return s_err != 0;
}

struct NoOp {
    __device__ void operator()() const {}
};

// InstState is rewritten by whichever block arrives last at a barrier, so every read of it bypasses L1.
__device__ __forceinline__ InstState load_state(const InstState* p) {
    static_assert(sizeof(InstState) % 8 == 0, "InstState layout");
    InstState s;
    const long long* src = reinterpret_cast<const long long*>(p);
    long long* dst = reinterpret_cast<long long*>(&s);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(InstState) / 8); ++k) dst[k] = __ldcg(src + k);
    return s;
}

// ---- SpMV over the rows of one tile -------------------------------------------------------------------------
// emit(row, value) receives y_row = sum_k A_rk x_k for every row of [r0, r1).
// L == 1: SELL-32, one thread per row (r0 is a multiple of 32). L >= 4: CSR with L lanes per row; emit runs
// on lane 0 of the row's group.
template <int L, typename VT, typename AT, typename Emit>
__device__ __forceinline__ void spmv_tile(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                          const VT* __restrict__ A, const VT* xin, int r0, int r1, Emit&& emit) {
    if constexpr (L == 1) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int s0 = r0 >> 5, s1 = (r1 + 31) >> 5;
        for (int s = s0 + warp; s < s1; s += kWarps) {
            const int base = __ldg(rp + s);
            const int w = (__ldg(rp + s + 1) - base) >> 5;
            const VT* av = A + base + lane;
            const int32_t* cv = ci + base + lane;
            AT acc = AT(0);
            int k = 0;
            for (; k + 8 <= w; k += 8) {
                VT v[8];
                int c[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    v[q] = __ldg(av + 32 * (k + q));
                    c[q] = __ldg(cv + 32 * (k + q));
                }
                VT x[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = ldcg(xin + c[q]);
#pragma unroll
                for (int q = 0; q < 8; ++q) acc = fma((AT)v[q], (AT)x[q], acc);
            }
            for (; k < w; ++k) acc = fma((AT)__ldg(av + 32 * k), (AT)ldcg(xin + __ldg(cv + 32 * k)), acc);
            const int row = (s << 5) + lane;
            if (row < r1) emit(row, acc);
        }
    } else {
        const int lane = threadIdx.x & (L - 1);
        const int grp = threadIdx.x / L, ngrp = kBlock / L;
        const unsigned mask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1)));
        for (int row = r0 + grp; row < r1; row += ngrp) {
            const int s = __ldg(rp + row), e = __ldg(rp + row + 1);
            AT acc = AT(0);
            for (int k = s + lane; k < e; k += L) acc = fma((AT)__ldg(A + k), (AT)ldcg(xin + __ldg(ci + k)), acc);
#pragma unroll
            for (int o = L / 2; o; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, L);
            if (lane == 0) emit(row, acc);
        }
    }
}

// ---- last-arriver reductions ---------------------------------------------------------------------------------

// Sum partial[q][t] over the tiles of every active instance for q in [0, NQ): the whole block when there is
// one instance, one warp per instance otherwise. Calls fn(i, sums) on one thread per instance.
template <int NQ, class Fn>
__device__ __forceinline__ void reduce_instances(const SolveArgs& a, Fn&& fn) {
    __shared__ double sm[NQ_ALL * 32];
    if (a.n_inst == 1) {
        double v[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] = 0.0;
        for (int t = threadIdx.x; t < a.n_tiles; t += kBlock)
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[q] += ldcg(a.partial + (size_t)q * a.n_tiles + t);
        block_sum<NQ>(v, sm);
        if (threadIdx.x == 0) fn(0, v);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < a.n_inst; i += kWarps) {
        if (!ldcg(&a.inst[i].active)) continue;
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
        if (lane == 0) fn(i, v);
    }
}

// Count active instances into bar->n_active (after the per-instance updates of this barrier).
__device__ __forceinline__ void count_active(const SolveArgs& a) {
    __syncthreads();
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int i = threadIdx.x; i < a.n_inst; i += kBlock) c += ldcg(&a.inst[i].active);
    if (c) atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) a.bar->n_active = cnt;
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

// FP64 CG update of one instance at a reduce point.
__device__ __forceinline__ void cg_update(InstState& st, double gamma, double rr, double delta, double tol2,
                                          int max_iter, bool count_iter) {
    const double bb = st.bb > 0.0 ? st.bb : 1.0;
    if (count_iter) st.iters += 1;
    st.relres = sqrt(rr / bb);
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
};

// ---- FP64 Chronopoulos-Gear Jacobi-PCG ----------------------------------------------------------------------

template <int L>
__global__ void __launch_bounds__(kBlock) k_cg64(SolveArgs a) {
    __shared__ double sm[NQ_ALL * 32];
    const int nt = a.n_tiles;
    const double tol2 = a.tol * a.tol;

    // init 1: r = b - A x, dinv, bb
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
        double v[1] = {0.0};
        spmv_tile<L, double, double>(a.rp, a.ci, a.A, a.x, r0, r1, [&](int row, double ax) {
            const double bi = a.b[row];
            a.r[row] = bi - ax;
            a.dinv[row] = 1.0 / a.A[a.diag[row]];
            v[0] += bi * bi;
        });
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
    if (grid_sync(a, NoOp{})) return;
    // init 3: w = A u; delta
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
        double v[1] = {0.0};
        spmv_tile<L, double, double>(a.rp, a.ci, a.A, a.u, r0, r1, [&](int row, double wu) {
            a.w[row] = wu;
            v[0] += wu * ldcg(a.u + row);
        });
        block_sum<1>(v, sm);
        if (threadIdx.x == 0) a.partial[(size_t)Q_DELTA * nt + t] = v[0];
    }
    if (grid_sync(a, [&] {
            reduce_instances<4>(a, [&](int i, double* s) {
                InstState st = load_state(a.inst + i);
                st.bb = s[Q_BB];
                st.first = 1;
                cg_update(st, s[Q_GAMMA], s[Q_RR], s[Q_DELTA], tol2, a.max_iter, false);
                a.inst[i] = st;
            });
            count_active(a);
        }))
        return;

    while (ldcg(&a.bar->n_active) > 0) {
        // phase A
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState* st = a.inst + a.tile_inst[t];
            if (!ldcg(&st->active)) continue;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[2] = {0.0, 0.0};
            CgRows<double> f{a.x,  a.r, a.u, a.w, a.p, a.s, a.dinv, ldcg(&st->alpha), ldcg(&st->beta),
                             ldcg(&st->first) != 0, v};
            for_rows<2>(r0, r1, f);
            block_sum<2>(v, sm);
            if (threadIdx.x == 0) {
                a.partial[(size_t)Q_GAMMA * nt + t] = v[0];
                a.partial[(size_t)Q_RR * nt + t] = v[1];
            }
        }
        if (grid_sync(a, NoOp{})) return;
        // phase B
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState* st = a.inst + a.tile_inst[t];
            if (!ldcg(&st->active)) continue;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[1] = {0.0};
            spmv_tile<L, double, double>(a.rp, a.ci, a.A, a.u, r0, r1, [&](int row, double wu) {
                a.w[row] = wu;
                v[0] = fma(wu, ldcg(a.u + row), v[0]);
            });
            block_sum<1>(v, sm);
            if (threadIdx.x == 0) a.partial[(size_t)Q_DELTA * nt + t] = v[0];
        }
        if (grid_sync(a, [&] {
                reduce_instances<3>(a, [&](int i, double* s) {
                    InstState st = load_state(a.inst + i);
                    st.first = 0;
                    cg_update(st, s[Q_GAMMA], s[Q_RR], s[Q_DELTA], tol2, a.max_iter, true);
                    a.inst[i] = st;
                });
                count_active(a);
            }))
            return;
    }

    // final: true residual ||b - A x|| for the reported relative residual
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
        double v[1] = {0.0};
        spmv_tile<L, double, double>(a.rp, a.ci, a.A, a.x, r0, r1, [&](int row, double ax) {
            const double ri = a.b[row] - ax;
            v[0] += ri * ri;
        });
        block_sum<1>(v, sm);
        if (threadIdx.x == 0) a.partial[(size_t)Q_RR * nt + t] = v[0];
    }
    grid_sync(a, [&] {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int i = warp; i < a.n_inst; i += kWarps) {
            double v = 0.0;
            for (int t = a.inst_t0[i] + lane; t < a.inst_t1[i]; t += 32) v += ldcg(a.partial + (size_t)Q_RR * nt + t);
#pragma unroll
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) {
                InstState st = load_state(a.inst + i);
                const double bb = st.bb > 0.0 ? st.bb : 1.0;
                st.relres = sqrt(v / bb);
                if (!isfinite(v) && st.status >= 0) st.status = RAFEM_ERR_NONFINITE;
                a.inst[i] = st;
            }
        }
    });
}

// ---- mixed precision: FP32 Chronopoulos-Gear inner iterations, FP64 residual refinement ---------------------

// Outer step of one row: r64 = b - A64 x; start the inner solve from d = 0 with r32 = r64.
struct OuterRow {
    const SolveArgs& a;
    double* v;  // [bb, rr64]
    float* f;   // [gamma, rr32]
    __device__ __forceinline__ void operator()(int row, double ax) const {
        const double bi = a.b[row];
        const double r64 = bi - ax;
        const float r32 = (float)r64;
        const float u32 = ldcg(a.dinv32 + row) * r32;
        a.r32[row] = r32;
        a.u32[row] = u32;
        a.d32[row] = 0.0f;
        v[0] = fma(bi, bi, v[0]);
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
__global__ void __launch_bounds__(kBlock) k_cg_mixed(SolveArgs a) {
    __shared__ double sm[NQ_ALL * 32];
    __shared__ float smf[NQ_ALL * 32];
    const int nt = a.n_tiles;
    const double tol2 = a.tol * a.tol;
    const double itol2 = a.inner_tol * a.inner_tol;

    // init: dinv32 from the FP32 diagonal (row-local; read again only by the same block after a barrier)
    for (int t = blockIdx.x; t < nt; t += gridDim.x)
        for (int i = a.tile_r0[t] + threadIdx.x; i < a.tile_r1[t]; i += kBlock) a.dinv32[i] = 1.0f / a.A32[a.diag[i]];
    __syncthreads();
    bool first_round = true;
    for (;;) {
        // ---------------- phase A ----------------
        if (!first_round) {
            for (int t = blockIdx.x; t < nt; t += gridDim.x) {
                const InstState* sp = a.inst + a.tile_inst[t];
                if (!ldcg(&sp->active)) continue;
                const int state = ldcg(&sp->outer);
                const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
                if (state == ST_OUTER) {
                    for_rows<4>(r0, r1, AddCorrection{a.x, a.d32});
                } else if (state == ST_ITER) {
                    float v[2] = {0.0f, 0.0f};
                    CgRows<float> f{a.d32, a.r32, a.u32, a.w32, a.p32, a.s32, a.dinv32, (float)ldcg(&sp->alpha),
                                    (float)ldcg(&sp->beta), ldcg(&sp->first) != 0, v};
                    for_rows<4>(r0, r1, f);
                    block_sum<2>(v, smf);
                    if (threadIdx.x == 0) {
                        a.partial[(size_t)Q_GAMMA * nt + t] = (double)v[0];
                        a.partial[(size_t)Q_RR * nt + t] = (double)v[1];
                    }
                }
            }
            if (grid_sync(a, NoOp{})) return;
        }
        // ---------------- phase B ----------------
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState* sp = a.inst + a.tile_inst[t];
            if (!ldcg(&sp->active)) continue;
            const int state = ldcg(&sp->outer);
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            if (state == ST_OUTER) {
                double v[2] = {0.0, 0.0};
                float f[2] = {0.0f, 0.0f};
                spmv_tile<L, double, double>(a.rp, a.ci, a.A, a.x, r0, r1, OuterRow{a, v, f});
                block_sum<2>(v, sm);
                block_sum<2>(f, smf);
                if (threadIdx.x == 0) {
                    a.partial[(size_t)Q_BB * nt + t] = v[0];
                    a.partial[(size_t)Q_RR64 * nt + t] = v[1];
                    a.partial[(size_t)Q_GAMMA * nt + t] = (double)f[0];
                    a.partial[(size_t)Q_RR * nt + t] = (double)f[1];
                }
            } else {
                float v[1] = {0.0f};
                spmv_tile<L, float, float>(a.rp, a.ci, a.A32, a.u32, r0, r1, [&](int row, float wu) {
                    a.w32[row] = wu;
                    v[0] = fmaf(wu, ldcg(a.u32 + row), v[0]);
                });
                block_sum<1>(v, smf);
                if (threadIdx.x == 0) a.partial[(size_t)Q_DELTA * nt + t] = (double)v[0];
            }
        }
        first_round = false;
        if (grid_sync(a, [&] {
                reduce_instances<NQ_ALL>(a, [&](int i, double* s) {
                    InstState st = load_state(a.inst + i);
                    if (st.outer == ST_OUTER) {
                        // FP64 residual of the current x: converged, capped, or start an inner solve
                        st.bb = s[Q_BB];
                        const double bb = st.bb > 0.0 ? st.bb : 1.0;
                        const double rr64 = s[Q_RR64];
                        st.relres = sqrt(rr64 / bb);
                        st.rr0 = rr64;  // outer residual at the start of this refinement
                        if (!isfinite(rr64)) {
                            stop(st, RAFEM_ERR_NONFINITE);
                        } else if (rr64 <= tol2 * bb) {
                            stop(st, RAFEM_OK);
                        } else if (st.refine >= a.max_refine || st.iters >= a.max_iter) {
                            stop(st, RAFEM_NOT_CONVERGED);
                        } else {
                            st.refine += 1;
                            st.outer = ST_START;
                            st.gamma = s[Q_GAMMA];  // inner gamma of the start vector
                            st.rr = s[Q_RR];        // inner ||r32||^2 at the start
                            st.first = 1;
                        }
                    } else if (st.outer == ST_START) {
                        st.first = 1;
                        if (!isfinite(s[Q_DELTA])) {
                            stop(st, RAFEM_ERR_NONFINITE);
                        } else if (cg_coefficients(st, st.gamma, s[Q_DELTA])) {
                            st.outer = ST_ITER;
                            st.rr_in0 = st.rr;
                        }
                    } else {
                        // ST_ITER: one inner FP32 iteration done
                        st.iters += 1;
                        st.first = 0;
                        const double rr = s[Q_RR];
                        st.rr = rr;
                        // stop the inner solve at inner_tol, or once the predicted outer residual
                        // ||r64|| * ||r32|| / ||r32_0|| is a quarter of the outer tolerance
                        const double bb = st.bb > 0.0 ? st.bb : 1.0;
                        const double target = fmax(itol2, 0.0625 * tol2 * bb / fmax(st.rr0, 1e-300));
                        if (!isfinite(rr) || !isfinite(s[Q_GAMMA]) || !isfinite(s[Q_DELTA])) {
                            stop(st, RAFEM_ERR_NONFINITE);
                        } else if (rr <= target * st.rr_in0 || st.iters >= a.max_iter) {
                            st.outer = ST_OUTER;
                        } else {
                            cg_coefficients(st, s[Q_GAMMA], s[Q_DELTA]);
                        }
                    }
                    a.inst[i] = st;
                });
                count_active(a);
            }))
            return;
        if (ldcg(&a.bar->n_active) == 0) break;
    }
}

__global__ void k_reset(InstState* inst, int n_inst, GridBarrier* bar) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
        InstState z = {};
        z.active = 1;
        z.first = 1;
        z.outer = ST_OUTER;
        inst[i] = z;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bar->count = 0;
        bar->err = 0;
        bar->n_active = n_inst;
    }
}

template <int L>
void* kernel_ptr(int precision) {
    return precision == RAFEM_PRECISION_MIXED ? (void*)k_cg_mixed<L> : (void*)k_cg64<L>;
}

void* select_kernel(int lanes, int precision) {
    switch (lanes) {
        case 1: return kernel_ptr<1>(precision);
        case 4: return kernel_ptr<4>(precision);
        case 8: return kernel_ptr<8>(precision);
        case 16: return kernel_ptr<16>(precision);
        case 32: return kernel_ptr<32>(precision);
        default: return nullptr;
    }
}

}  // namespace

int krylov_max_blocks(int lanes, int precision, int* block_threads) {
    void* k = select_kernel(lanes, precision);
    if (!k) return 0;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlock, 0) != cudaSuccess) return 0;
    if (block_threads) *block_threads = kBlock;
    return per_sm * sms;
}

cudaError_t launch_krylov(const SolveArgs& a, int lanes, int precision, int grid, int block, cudaStream_t st) {
    void* k = select_kernel(lanes, precision);
    if (!k) return cudaErrorInvalidValue;
    k_reset<<<(a.n_inst + 255) / 256, 256, 0, st>>>(a.inst, a.n_inst, a.bar);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
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
