// Persistent restarted GMRES(m) (FP64) with right Jacobi preconditioning on the SELL-32 layout.
//
// Sec. III-B solves every corrector pass's system with a restarted GMRES(m) to a 1e-10 residual, m tuned per mesh;
// Sec. II-B: GMRES suits general (nonsymmetric) systems. Here one cooperative launch runs all cycles:
//   cycle start (SpMV):  r = b - A x, partial (r, r)                                   -- barrier: beta = ||r|| --
//   Arnoldi step j, with u the unnormalised new basis vector and s its norm (r, beta for j = 0):
//     S (SpMV):   v_j = u / s (own rows),  w = A M^-1 u / s,  partials h_ij = (w, v_i), i <= j       -- barrier --
//     O1:         w -= sum_i h_ij v_i,  partials c_ij = (w, v_i)                                    -- barrier --
//     O2:         w -= sum_i c_ij v_i,  h_ij += c_ij,  partial (w, w)      -- barrier: h_{j+1,j} = ||w|| --
//   (classical Gram-Schmidt with one reorthogonalisation); every block applies the Givens rotations to column j
//   of the Hessenberg matrix in shared memory (same inputs, same bits) and reads the residual estimate |g_{j+1}|.
//   cycle end:    y = R^-1 g (back substitution),  x += M^-1 sum_i y_i v_i (own rows)              -- barrier --
// The cycle restarts until the true residual of a cycle start meets the tolerance. Dots are reduced per warp with
// shuffles, per block in shared memory and across blocks in a fixed order (deterministic). Every barrier wait is
// bounded.
#include <cuda_runtime.h>

#include <cmath>

#include "grid_sync.cuh"
#include "internal.h"

namespace rafem {

namespace {

constexpr int kBlock = 512;
constexpr int kWarps = kBlock / 32;
constexpr int kBatch = 8;

struct Args {
    int N, m;
    const int32_t* sp;
    const int32_t* sc;
    const int16_t* sc16;
    const double* A;
    const int32_t* diag;
    const double* b;
    double* x;
    double* Vb;       // [m][N] basis
    double* w[2];     // [N] alternating unnormalised vectors
    double* dinv;     // [N]
    double* partial;  // [2 (m + 1) + 2][grid]
    GridBarrier* bar;
    InstState* inst;
    double tol;
    int max_iter;
    long long spin_limit_ns;
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

template <class Fn>
__device__ __forceinline__ void for_slices(int S, const Fn& f) {
    const int tw = gridDim.x * kWarps;
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * kWarps + (threadIdx.x >> 5); s < S; s += tw) f(s, s * 32 + lane);
}

// sum_k A_row,k dinv_k u_k (dinv = null: plain A u)
__device__ __forceinline__ double spmv_row(const Args& a, const double* u, const double* dinv, int s, int row) {
    const int lane = row & 31;
    const int base = __ldg(a.sp + s), w = (__ldg(a.sp + s + 1) - base) >> 5;
    double acc = 0.0;
    for (int k = 0; k < w; k += kBatch) {
        double m[kBatch], y[kBatch];
        int c[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            const int pos = base + 32 * (k + t) + lane;
            const bool ok = k + t < w;
            m[t] = ok ? __ldg(a.A + pos) : 0.0;
            c[t] = ok ? (a.sc16 ? row + (int)__ldg(a.sc16 + pos) : __ldg(a.sc + pos)) : -1;
        }
        // dinv is written in this launch, so it is read through L2 like the vectors
#pragma unroll
        for (int t = 0; t < kBatch; ++t)
            y[t] = c[t] >= 0 ? (dinv ? ldcg(u + c[t]) * ldcg(dinv + c[t]) : ldcg(u + c[t])) : 0.0;
#pragma unroll
        for (int t = 0; t < kBatch; ++t) acc = fma(m[t], y[t], acc);
    }
    return acc;
}

// Per-warp accumulation of up to n dot products into shared memory acc[warp][i] (lane 0 adds each warp sum).
__device__ __forceinline__ void warp_add(double* acc, int i, double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) acc[(threadIdx.x >> 5) * 72 + i] += v;
}

// Block sums of the n per-warp accumulators -> partial[i][blockIdx.x]; accumulators cleared for the next phase.
__device__ __forceinline__ void publish(double* acc, int n, double* part) {
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int wp = 0; wp < kWarps; ++wp) s += acc[wp * 72 + i];
        part[(size_t)i * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWarps * 72; i += blockDim.x) acc[i] = 0.0;
}

// After a barrier: tot[i] = sum over blocks of partial[i][.] (fixed order; warp per quantity).
__device__ __forceinline__ void totals(const double* part, int n, double* tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < n; i += kWarps) {
        double s = 0.0;
        for (int t = lane; t < (int)gridDim.x; t += 32) s += ldcg(part + (size_t)i * gridDim.x + t);
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) tot[i] = s;
    }
    __syncthreads();
}

// acc[warp][i] += (w, v_i) over this warp's rows for i < n. Each lane keeps kDot running sums in registers over
// all its rows and the warp reduces them once per group of kDot basis vectors (a warp reduction per row and
// vector would serialise the warp on shuffle latency). w holds values this thread wrote itself.
constexpr int kDot = 8;
__device__ __forceinline__ void dots(const Args& a, double* acc, const double* w, int n, int S) {
    for (int i0 = 0; i0 < n; i0 += kDot) {
        double sum[kDot];
#pragma unroll
        for (int t = 0; t < kDot; ++t) sum[t] = 0.0;
        for_slices(S, [&](int, int row) {
            if (row >= a.N) return;
            const double wi = w[row];
#pragma unroll
            for (int t = 0; t < kDot; ++t)
                if (i0 + t < n) sum[t] = fma(wi, ldcg(a.Vb + (size_t)(i0 + t) * a.N + row), sum[t]);
        });
#pragma unroll
        for (int t = 0; t < kDot; ++t)
            if (i0 + t < n) warp_add(acc, i0 + t, sum[t]);
    }
}

__global__ void __launch_bounds__(kBlock, 1) k_gmres(Args a) {
    extern __shared__ double smem[];
    // layout: acc [kWarps][72] | H [(m+1) x m] column-major | cs[m] | sn[m] | g[m+1] | tot[72] | y[m]
    const int m = a.m;
    double* acc = smem;
    double* H = acc + kWarps * 72;
    double* cs = H + (size_t)(m + 1) * m;
    double* sn = cs + m;
    double* g = sn + m;
    double* tot = g + (m + 1);
    double* yv = tot + 72;
    for (int i = threadIdx.x; i < kWarps * 72; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    // partial-sum buffers of consecutive phases are disjoint: S -> PA, O1 -> PB, O2 -> PC, cycle start -> PD
    const size_t G = gridDim.x;
    double* PA = a.partial;
    double* PB = PA + (size_t)(m + 1) * G;
    double* PC = PB + (size_t)(m + 1) * G;
    double* PD = PC + G;
    const int N = a.N, S = (N + 31) / 32;
    unsigned target = 0;
    bool err = false;
    int iters = 0, status = RAFEM_NOT_CONVERGED, cycles = 0;
    double bb = 0.0, rr = 0.0;
    // dinv = 1 / diag(A); (b, b)
    {
        double v = 0.0;
        for_slices(S, [&](int, int row) {
            if (row < N) {
                a.dinv[row] = 1.0 / __ldg(a.A + __ldg(a.diag + row));
                v = fma(a.b[row], a.b[row], v);
            }
        });
        warp_add(acc, 0, v);
        publish(acc, 1, PD);
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        totals(PD, 1, tot);
        bb = tot[0];
    }
    const double thr = a.tol * a.tol * (bb > 0.0 ? bb : 1.0);
    while (!err) {
        // cycle start: r = b - A x into w[0], (r, r)
        {
            double v = 0.0;
            for_slices(S, [&](int s, int row) {
                if (row >= N) return;
                const double ri = a.b[row] - spmv_row(a, a.x, nullptr, s, row);
                a.w[0][row] = ri;
                v = fma(ri, ri, v);
            });
            warp_add(acc, 0, v);
            publish(acc, 1, PD);
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals(PD, 1, tot);
            rr = tot[0];
        }
        if (!(rr == rr)) { status = RAFEM_ERR_NONFINITE; break; }
        if (rr <= thr) { status = RAFEM_OK; break; }
        if (iters >= a.max_iter) break;
        ++cycles;
        if (threadIdx.x == 0) {
            g[0] = sqrt(rr);
            for (int i = 1; i <= m; ++i) g[i] = 0.0;
        }
        __syncthreads();
        double scale = sqrt(rr);  // norm of the unnormalised vector held in w[cur]
        int cur = 0, k = 0;
        for (int j = 0; j < m; ++j) {
            const double* u = a.w[cur];
            double* wn = a.w[cur ^ 1];
            double* vj = a.Vb + (size_t)j * N;
            const double inv = 1.0 / scale;
            // S: v_j = u / s, w = A M^-1 u / s, then h_ij = (w, v_i) for i <= j
            for_slices(S, [&](int s, int row) {
                if (row >= N) return;
                wn[row] = spmv_row(a, u, a.dinv, s, row) * inv;
                vj[row] = ldcg(u + row) * inv;
            });
            dots(a, acc, wn, j + 1, S);
            publish(acc, j + 1, PA);
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals(PA, j + 1, tot);
            for (int i = threadIdx.x; i <= j; i += blockDim.x) H[(size_t)j * (m + 1) + i] = tot[i];
            __syncthreads();
            // O1: w -= sum_i h_ij v_i, then c_ij = (w, v_i)
            for_slices(S, [&](int, int row) {
                if (row >= N) return;
                double wi = wn[row];
                for (int i = 0; i <= j; ++i)
                    wi = fma(-H[(size_t)j * (m + 1) + i], ldcg(a.Vb + (size_t)i * N + row), wi);
                wn[row] = wi;
            });
            dots(a, acc, wn, j + 1, S);
            publish(acc, j + 1, PB);
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals(PB, j + 1, tot);
            // O2: w -= sum_i c_ij v_i, h_ij += c_ij, (w, w)
            {
                double v = 0.0;
                for_slices(S, [&](int, int row) {
                    if (row >= N) return;
                    double wi = wn[row];
                    for (int i = 0; i <= j; ++i) wi = fma(-tot[i], ldcg(a.Vb + (size_t)i * N + row), wi);
                    wn[row] = wi;
                    v = fma(wi, wi, v);
                });
                __syncthreads();
                for (int i = threadIdx.x; i <= j; i += blockDim.x) H[(size_t)j * (m + 1) + i] += tot[i];
                warp_add(acc, 0, v);
                publish(acc, 1, PC);
                if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
                totals(PC, 1, tot);
            }
            const double hn = sqrt(tot[0]);
            // Givens rotations on column j (thread 0; every block computes the same bits)
            if (threadIdx.x == 0) {
                double* col = H + (size_t)j * (m + 1);
                col[j + 1] = hn;
                for (int i = 0; i < j; ++i) {
                    const double t0 = cs[i] * col[i] + sn[i] * col[i + 1];
                    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
                    col[i] = t0;
                }
                const double den = hypot(col[j], col[j + 1]);
                const double c = den > 0.0 ? col[j] / den : 1.0, sv = den > 0.0 ? col[j + 1] / den : 0.0;
                cs[j] = c;
                sn[j] = sv;
                col[j] = den;
                col[j + 1] = 0.0;
                g[j + 1] = -sv * g[j];
                g[j] = c * g[j];
            }
            __syncthreads();
            ++iters;
            k = j + 1;
            scale = hn;
            cur ^= 1;
            if (g[j + 1] * g[j + 1] <= thr || !(hn > 0.0) || iters >= a.max_iter) break;
        }
        if (err) break;
        // y = R^-1 g, x += M^-1 sum_i y_i v_i
        if (threadIdx.x == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double t = g[i];
                for (int l = i + 1; l < k; ++l) t -= H[(size_t)l * (m + 1) + i] * yv[l];
                const double d = H[(size_t)i * (m + 1) + i];
                yv[i] = d != 0.0 ? t / d : 0.0;
            }
        }
        __syncthreads();
        for_slices(S, [&](int, int row) {
            if (row >= N) return;
            double t = 0.0;
            for (int i = 0; i < k; ++i) t = fma(yv[i], ldcg(a.Vb + (size_t)i * N + row), t);
            a.x[row] = fma(a.dinv[row], t, a.x[row]);
        });
        if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        InstState st = {};
        st.bb = bb;
        st.rr = rr;
        st.iters = iters;
        st.refine = cycles;
        st.status = err ? (a.bar->err ? a.bar->err : RAFEM_ERR_TIMEOUT) : status;
        st.relres = sqrt(rr / (bb > 0.0 ? bb : 1.0));
        a.inst[0] = st;
    }
}

size_t smem_bytes(int m) {
    return sizeof(double) * ((size_t)kWarps * 72 + (size_t)(m + 1) * m + m + m + (m + 1) + 72 + m);
}

}  // namespace

int gmres_max_blocks(int m) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const size_t sh = smem_bytes(m);
    if (cudaFuncSetAttribute(k_gmres, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_gmres, kBlock, sh) != cudaSuccess) return 0;
    return sms * (per < 1 ? per : 1);
}

cudaError_t launch_gmres(const GmresArgs& s, int grid, cudaStream_t st) {
    Args a{s.N, s.m, s.sp, s.sc, s.sc16, s.A, s.diag, s.b, s.x, s.V, {s.w0, s.w1}, s.dinv, s.partial, s.bar,
           s.inst, s.tol, s.max_iter, s.spin_limit_ns};
    cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    if (s.bar_missing > 0 && (e = launch_barrier_reset(s.bar, s.bar_missing, st)) != cudaSuccess) return e;
    void* params[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_gmres, dim3(grid), dim3(kBlock), params, smem_bytes(s.m), st);
}

}  // namespace rafem
