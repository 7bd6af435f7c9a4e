// Persistent fused Krylov solvers: one cooperative launch runs a whole solve (all iterations) on the device.
//
// The paper solves each corrector pass's global system with library solvers (GMRES(m) to 1e-10 residual,
// Sec. III-B) and moves vector reductions to thrust (Sec. III-A). For the symmetric positive-definite lifted
// systems here, CG is the method of choice (Sec. II-B); it runs as one persistent kernel whose phases are
// separated by grid barriers, with every dot product fused into the phase that produces its operands:
//
//   Chronopoulos-Gear preconditioned CG (two grid barriers per iteration instead of three):
//     phase V (row-local):  p = u + beta p,  s = w + beta s,  x += alpha p,  r -= alpha s,  u = M^-1 r,
//                           partial sums of gamma = (r, u) and rr = (r, r)
//     -- barrier --
//     phase S (SpMV):       w = A u,  partial sum of delta = (w, u)
//     -- barrier; the last block to arrive reduces the partial sums (fixed order: deterministic) and sets
//        beta = gamma / gamma_prev, alpha = gamma / (delta - beta gamma / alpha_prev) per instance --
//
// Work is split into tiles (contiguous row ranges, each belonging to one problem instance); blocks stride over
// tiles, and instances that have converged are skipped, so many independent systems of different sizes run
// in one launch (the batching form) with per-instance convergence.
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

enum { Q_GAMMA = 0, Q_RR = 1, Q_DELTA = 2, Q_BB = 3 };

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

struct NoOp {
    __device__ void operator()() const {}
};

// y_row = sum_k A[k] x[ci[k]] with L lanes per row; emit(row, value) runs on lane 0 of the row's group.
template <int L, typename VT, typename AT, typename Emit>
__device__ __forceinline__ void spmv_tile(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                          const VT* __restrict__ A, const VT* xin, int r0, int r1, Emit&& emit) {
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

// ---- last-arriver reductions ---------------------------------------------------------------------------------

// Sum partial[q][t] over the tiles of instance i, for q in [0, NQ). Whole block when there is one instance,
// one warp per instance otherwise. Calls fn(i, sums) on one thread per instance.
template <int NQ, class Fn>
__device__ __forceinline__ void reduce_instances(const SolveArgs& a, Fn&& fn) {
    __shared__ double sm[4 * 32];
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

// CG scalar update of one instance from gamma, rr, delta; returns nothing, writes InstState.
__device__ __forceinline__ void cg_update(InstState& st, double gamma, double rr, double delta, double tol2,
                                          int max_iter, bool count_iter) {
    const double bb = st.bb > 0.0 ? st.bb : 1.0;
    if (count_iter) st.iters += 1;
    st.relres = sqrt(rr / bb);
    st.rr = rr;
    if (!isfinite(gamma) || !isfinite(rr) || !isfinite(delta)) {
        st.status = RAFEM_ERR_NONFINITE;
        st.active = 0;
        return;
    }
    if (rr <= tol2 * bb) {
        st.status = RAFEM_OK;
        st.active = 0;
        return;
    }
    if (st.iters >= max_iter) {
        st.status = RAFEM_NOT_CONVERGED;
        st.active = 0;
        return;
    }
    double alpha, beta;
    if (st.first) {
        beta = 0.0;
        alpha = gamma / delta;
        if (!(delta > 0.0) || !(gamma > 0.0)) {
            st.status = RAFEM_ERR_BREAKDOWN;
            st.active = 0;
            return;
        }
    } else {
        beta = gamma / st.gamma_prev;
        const double den = delta - beta * gamma / st.alpha_prev;
        if (!(den > 0.0) || !(gamma > 0.0)) {
            st.status = RAFEM_ERR_BREAKDOWN;
            st.active = 0;
            return;
        }
        alpha = gamma / den;
    }
    st.alpha = alpha;
    st.beta = beta;
    st.gamma_prev = gamma;
    st.alpha_prev = alpha;
}

// ---- FP64 Chronopoulos-Gear Jacobi-PCG ----------------------------------------------------------------------

template <int L>
__global__ void __launch_bounds__(kBlock) k_cg64(SolveArgs a) {
    __shared__ double sm[4 * 32];
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
    // init 2 needs only row-local data of init 1 (same tiles, same block): u = dinv r; gamma, rr
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
        // phase V
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState* st = a.inst + a.tile_inst[t];
            if (!ldcg(&st->active)) continue;
            const double alpha = ldcg(&st->alpha), beta = ldcg(&st->beta);
            const bool first = ldcg(&st->first) != 0;
            const int r0 = a.tile_r0[t], r1 = a.tile_r1[t];
            double v[2] = {0.0, 0.0};
            for (int i = r0 + threadIdx.x; i < r1; i += kBlock) {
                const double ui = ldcg(a.u + i), wi = ldcg(a.w + i);
                const double pi = first ? ui : fma(beta, ldcg(a.p + i), ui);
                const double si = first ? wi : fma(beta, ldcg(a.s + i), wi);
                a.p[i] = pi;
                a.s[i] = si;
                a.x[i] = fma(alpha, pi, ldcg(a.x + i));
                const double ri = fma(-alpha, si, ldcg(a.r + i));
                a.r[i] = ri;
                const double un = ldcg(a.dinv + i) * ri;
                a.u[i] = un;
                v[0] += ri * un;
                v[1] += ri * ri;
            }
            block_sum<2>(v, sm);
            if (threadIdx.x == 0) {
                a.partial[(size_t)Q_GAMMA * nt + t] = v[0];
                a.partial[(size_t)Q_RR * nt + t] = v[1];
            }
        }
        if (grid_sync(a, NoOp{})) return;
        // phase S
        for (int t = blockIdx.x; t < nt; t += gridDim.x) {
            const InstState* st = a.inst + a.tile_inst[t];
            if (!ldcg(&st->active)) continue;
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

__global__ void k_reset(InstState* inst, int n_inst, GridBarrier* bar) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
        InstState z = {};
        z.active = 1;
        z.first = 1;
        z.outer = 1;
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
    (void)precision;
    return (void*)k_cg64<L>;
}

void* select_kernel(int lanes, int precision) {
    switch (lanes) {
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
    k_reset<<<(a.n_inst + 255) / 256, 256, 0, st>>>(a.inst, a.n_inst, a.bar);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SolveArgs copy = a;
    void* args[] = {&copy};
    return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace rafem
