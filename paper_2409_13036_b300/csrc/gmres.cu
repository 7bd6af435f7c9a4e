// Persistent restarted GMRES(m) (FP64) with right Jacobi preconditioning on the SELL-32 layout.
//
// Sec. III-B solves every corrector pass's system with a restarted GMRES(m) to a 1e-10 residual, m tuned per mesh,
// and notes that an m adapted during the simulation and for each solution would reduce the stagnation it observes;
// Sec. II-B: GMRES suits general (nonsymmetric) systems. Here one cooperative launch runs all cycles:
//   cycle start (SpMV):  r = b - A x, partial (r, r)                                   -- barrier: beta = ||r|| --
//   Arnoldi step j, with u the unnormalised new basis vector and s its norm (r, beta for j = 0):
//     S (SpMV):   v_j = u / s (own rows),  w = A M^-1 u / s,
//                 partials h_ij = (w, v_i), i <= j, and (w, w)                                       -- barrier --
//     then, by Pythagoras, ||w - sum_i h_ij v_i||^2 = (w, w) - sum_i h_ij^2. While that keeps at least half of
//     (w, w) the cancellation is mild and the norm is accurate, so one pass suffices:
//     O:          w -= sum_i h_ij v_i                                    -- barrier (before the next SpMV) --
//     otherwise classical Gram-Schmidt is repeated once ("twice is enough", Kahan-Parlett):
//     O1:         w -= sum_i h_ij v_i,  partials c_ij = (w, v_i), (w, w)                            -- barrier --
//     O2:         w -= sum_i c_ij v_i,  h_ij += c_ij,  ||w||^2 = (w, w) - sum_i c_ij^2            -- barrier --
//   Every block applies the Givens rotations to column j of the Hessenberg matrix in shared memory (same inputs,
//   same bits) and reads the residual estimate |g_{j+1}|; the step that reaches the tolerance or ends the cycle
//   skips its O phase (w is not needed).
//   cycle end:    y = R^-1 g (back substitution),  x += M^-1 sum_i y_i v_i (own rows)              -- barrier --
// The cycle restarts until the true residual of a cycle start meets the tolerance.
//
// Restart length. With m_min > 0 the length of each cycle adapts between m_min and m (the allocated basis) by the
// rule of Baker, Jessup and Kolev, "A simple strategy for varying the restart parameter in GMRES(m)", J. Comput.
// Appl. Math. 230 (2009): with cr the ratio of the true residual norms at the start of this cycle and the last,
// cr > cos(8 deg) (stagnation) sets m; cr < cos(80 deg) (fast) keeps the length; otherwise the length drops by 3,
// back to m once it would fall below m_min. The length a solve ends with starts the next solve of the same system
// (the simulation's solves adapt too). Stagnation handling: cycles at the full length m that reduce the residual
// by less than 0.1% are counted, and two in a row end the solve (RAFEM_NOT_CONVERGED) instead of burning the
// iteration cap: at that rate a reduction of 1e-10 would take more than 23,000 cycles.
// Dots are reduced per warp with shuffles, per block in shared memory and across blocks in a fixed order
// (deterministic). Every barrier wait is bounded.
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
    int N, m, m_min;        // basis size (the longest cycle); shortest adaptive cycle (0: every cycle has m steps)
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
    int32_t* m_state;       // adaptive length the next solve starts with (read at launch, written at the end)
};

// Restart-length rule (Baker, Jessup, Kolev 2009): thresholds on the cycle's convergence ratio and the decrement.
constexpr double kMaxCr = 0.99026806874157031;   // cos(8 deg)
constexpr double kMinCr = 0.17364817766693041;   // cos(80 deg)
constexpr int kDecrement = 3;
constexpr double kStagnant = 0.999;              // a full-length cycle keeping 99.9% of the residual is stagnant
constexpr int kStagnantStop = 2;                 // consecutive stagnant full-length cycles that end the solve

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
// self: also (w, w) into acc[.][n], accumulated in the first group's pass over the rows.
__device__ __forceinline__ void dots(const Args& a, double* acc, const double* w, int n, int S, bool self = false) {
    for (int i0 = 0; i0 < n; i0 += kDot) {
        double sum[kDot], ww = 0.0;
#pragma unroll
        for (int t = 0; t < kDot; ++t) sum[t] = 0.0;
        const bool with_self = self && i0 == 0;
        for_slices(S, [&](int, int row) {
            if (row >= a.N) return;
            const double wi = w[row];
            if (with_self) ww = fma(wi, wi, ww);
#pragma unroll
            for (int t = 0; t < kDot; ++t)
                if (i0 + t < n) sum[t] = fma(wi, ldcg(a.Vb + (size_t)(i0 + t) * a.N + row), sum[t]);
        });
#pragma unroll
        for (int t = 0; t < kDot; ++t)
            if (i0 + t < n) warp_add(acc, i0 + t, sum[t]);
        if (with_self) warp_add(acc, n, ww);
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
    // restart length of the current cycle (adaptive: from the previous solve of this system)
    int m_cur = m;
    if (a.m_min > 0 && a.m_state) m_cur = min(max(*(volatile int32_t*)a.m_state, a.m_min), m);
    double rr_prev = -1.0;
    int stagnant = 0, reorths = 0;
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
        if (rr_prev > 0.0) {
            // the last cycle's convergence ratio decides this cycle's length (every block: same bits)
            const double cr = sqrt(rr / rr_prev);
            if (m_cur == m && cr > kStagnant) {
                if (++stagnant >= kStagnantStop) break;  // stagnated at the full length: NOT_CONVERGED
            } else {
                stagnant = 0;
            }
            if (a.m_min > 0) {
                if (cr > kMaxCr)
                    m_cur = m;
                else if (cr >= kMinCr)
                    m_cur = m_cur - kDecrement >= a.m_min ? m_cur - kDecrement : m;
            }
        }
        rr_prev = rr;
        ++cycles;
        if (threadIdx.x == 0) {
            g[0] = sqrt(rr);
            for (int i = 1; i <= m; ++i) g[i] = 0.0;
        }
        __syncthreads();
        double scale = sqrt(rr);  // norm of the unnormalised vector held in w[cur]
        int cur = 0, k = 0;
        for (int j = 0; j < m_cur; ++j) {
            const double* u = a.w[cur];
            double* wn = a.w[cur ^ 1];
            double* vj = a.Vb + (size_t)j * N;
            double* Hj = H + (size_t)j * (m + 1);
            const double inv = 1.0 / scale;
            // S: v_j = u / s, w = A M^-1 u / s, then h_ij = (w, v_i) for i <= j and (w, w)
            for_slices(S, [&](int s, int row) {
                if (row >= N) return;
                wn[row] = spmv_row(a, u, a.dinv, s, row) * inv;
                vj[row] = ldcg(u + row) * inv;
            });
            dots(a, acc, wn, j + 1, S, true);
            publish(acc, j + 2, PA);
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals(PA, j + 2, tot);
            double proj = 0.0;  // sum_i h_ij^2 (same order in every block)
            for (int i = 0; i <= j; ++i) proj = fma(tot[i], tot[i], proj);
            const double ww = tot[j + 1];
            double nh2 = ww - proj;
            const bool reorth = !(nh2 >= 0.5 * ww);
            for (int i = threadIdx.x; i <= j; i += blockDim.x) Hj[i] = tot[i];
            __syncthreads();
            if (reorth) {
                ++reorths;
                // O1: w -= sum_i h_ij v_i, then c_ij = (w, v_i) and (w, w)
                for_slices(S, [&](int, int row) {
                    if (row >= N) return;
                    double wi = wn[row];
                    for (int i = 0; i <= j; ++i) wi = fma(-Hj[i], ldcg(a.Vb + (size_t)i * N + row), wi);
                    wn[row] = wi;
                });
                dots(a, acc, wn, j + 1, S, true);
                publish(acc, j + 2, PB);
                if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
                totals(PB, j + 2, tot);
                double c2 = 0.0;
                for (int i = 0; i <= j; ++i) c2 = fma(tot[i], tot[i], c2);
                nh2 = tot[j + 1] - c2;
                for (int i = threadIdx.x; i <= j; i += blockDim.x) Hj[i] += tot[i];
                __syncthreads();
            }
            const double hn = sqrt(fmax(nh2, 0.0));
            // Givens rotations on column j (thread 0; every block computes the same bits)
            if (threadIdx.x == 0) {
                Hj[j + 1] = hn;
                for (int i = 0; i < j; ++i) {
                    const double t0 = cs[i] * Hj[i] + sn[i] * Hj[i + 1];
                    Hj[i + 1] = -sn[i] * Hj[i] + cs[i] * Hj[i + 1];
                    Hj[i] = t0;
                }
                const double den = hypot(Hj[j], Hj[j + 1]);
                const double c = den > 0.0 ? Hj[j] / den : 1.0, sv = den > 0.0 ? Hj[j + 1] / den : 0.0;
                cs[j] = c;
                sn[j] = sv;
                Hj[j] = den;
                Hj[j + 1] = 0.0;
                g[j + 1] = -sv * g[j];
                g[j] = c * g[j];
            }
            __syncthreads();
            ++iters;
            k = j + 1;
            if (g[j + 1] * g[j + 1] <= thr || !(hn > 0.0) || iters >= a.max_iter || j + 1 == m_cur) break;
            // O (or O2): the next basis vector, unnormalised; its norm hn is already known. tot holds the h_ij of
            // the single pass, or the c_ij of the second pass.
            for_slices(S, [&](int, int row) {
                if (row >= N) return;
                double wi = wn[row];
                for (int i = 0; i <= j; ++i) wi = fma(-tot[i], ldcg(a.Vb + (size_t)i * N + row), wi);
                wn[row] = wi;
            });
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            scale = hn;
            cur ^= 1;
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
    if (a.m_state && blockIdx.x == 0 && threadIdx.x == 0) *a.m_state = m_cur;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        InstState st = {};
        st.bb = bb;
        st.rr = rr;
        st.iters = iters;
        st.refine = cycles;
        st.breakdowns = reorths;  // Arnoldi steps that needed the second Gram-Schmidt pass
        st.outer = m_cur;         // restart length of the last cycle
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
    Args a{s.N, s.m, s.m_min, s.sp, s.sc, s.sc16, s.A, s.diag, s.b, s.x, s.V, {s.w0, s.w1}, s.dinv, s.partial, s.bar,
           s.inst, s.tol, s.max_iter, s.spin_limit_ns, s.m_state};
    cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    if (s.bar_missing > 0 && (e = launch_barrier_reset(s.bar, s.bar_missing, st)) != cudaSuccess) return e;
    void* params[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_gmres, dim3(grid), dim3(kBlock), params, smem_bytes(s.m), st);
}

}  // namespace rafem
