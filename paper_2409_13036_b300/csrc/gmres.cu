// Persistent restarted GMRES(m) (FP64) with right Jacobi preconditioning on the SELL-32 layout.
//
// Sec. III-B solves every corrector pass's system with a restarted GMRES(m) to a 1e-10 residual, m tuned per mesh,
// and notes that an m adapted during the simulation and for each solution would reduce the stagnation it observes;
// Sec. II-B: GMRES suits general (nonsymmetric) systems. Here one cooperative launch runs all cycles:
//   cycle start (SpMV):  r = b - A x, partial (r, r)                                   -- barrier: beta = ||r|| --
//   Arnoldi step j, with u the unnormalised new basis vector and s its norm (r, beta for j = 0):
//     S (SpMV):   v_j = u / s (own rows),  w = A M^-1 u / s,
//                 partials h_ij = (w, v_i), i <= j, and (w, w)                                       -- barrier --
//     then, by Pythagoras, ||w - sum_i h_ij v_i||^2 = (w, w) - sum_i h_ij^2. While that keeps at least 1% of
//     (w, w) (the new direction at least a tenth of w's norm) one pass suffices: each restart recomputes the true
//     residual, so weaker orthogonality could only cost Arnoldi steps, and on the potential systems it costs none
//     (a rule at half of (w, w) took the second pass at every step, 35% of the solve, for the same step counts):
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
// back to m once it would fall below m_min; every solve starts at m (carrying a short length over to the next
// solve of the simulation cost more cycles on the measured workloads than it saved). Stagnation handling: cycles at the full length m that reduce the residual
// by less than 0.1% are counted, and two in a row end the solve (RAFEM_NOT_CONVERGED) instead of burning the
// iteration cap: at that rate a reduction of 1e-10 would take more than 23,000 cycles.
//
// Layout of the work: block b owns the rows [b R, (b + 1) R) (R a multiple of 32, one tile per block) in every
// phase, so row-local vectors stay with their block. The SpMVs stream the matrix through the shared-memory ring of
// the CG kernels (bulk copies by a producer warp, sell_ring.cuh) and gather z = M^-1 u, which the phase before
// each SpMV writes for its own rows. The passes over the basis are row-local and vectorised: each thread takes
// two consecutive rows (16-byte loads) and up to four basis vectors per batch, so every thread has five
// independent loads in flight. The basis is stored with a row stride rounded up to a multiple of 32.
// Dots are reduced per warp with shuffles, per block in shared memory and across blocks in a fixed order
// (deterministic). Every wait is bounded.
#include <cuda_runtime.h>

#include <cmath>

#include "grid_sync.cuh"
#include "internal.h"
#include "dw.cuh"
#include "sell_ring.cuh"

namespace rafem {

namespace {

using namespace sell;

constexpr int kAcc = 72;  // per-warp accumulator slots: up to 64 dots + (w, w)

struct Args {
    int N, m, m_min;        // basis size (the longest cycle); shortest adaptive cycle (0: every cycle has m steps)
    int ld;                 // row stride of the basis (N rounded up to a multiple of 32)
    const int32_t* sp;
    const int32_t* sc;
    const int16_t* sc16;
    const int32_t* pat_off;   // one column pattern per slice (kernel code 3), or null
    const int32_t* pat_pool;
    const double* A;
    const int32_t* diag;
    const double* b;
    double* x;
    float2* Vb;       // [m][ld] basis, double-word (float pairs, 8 bytes per entry like the double it replaces)
    double* w[2];     // [N] alternating unnormalised vectors
    double* z;        // [N] M^-1 of the vector the next SpMV multiplies
    double* dinv;     // [N]
    double* H;        // [grid][(m + 1) m] Hessenberg matrix, one copy per block (column-major)
    double* partial;  // [2 (m + 2) + 2][grid]
    GridBarrier* bar;
    InstState* inst;
    double tol;
    int max_iter;
    long long spin_limit_ns;
};

// Restart-length rule (Baker, Jessup, Kolev 2009): thresholds on the cycle's convergence ratio and the decrement.
constexpr double kMaxCr = 0.99026806874157031;   // cos(8 deg)
constexpr double kMinCr = 0.17364817766693041;   // cos(80 deg)
constexpr int kDecrement = 3;
constexpr double kStagnant = 0.999;              // a full-length cycle keeping 99.9% of the residual is stagnant
constexpr int kStagnantStop = 2;                 // consecutive stagnant full-length cycles that end the solve
constexpr double kReorth = 0.01;                 // second Gram-Schmidt pass when the first keeps < 1% of (w, w)

// Per-warp accumulation into shared memory acc[warp][i] (lane 0 adds the warp's sum).
__device__ __forceinline__ void warp_add(double* acc, int i, double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) acc[(threadIdx.x >> 5) * kAcc + i] += v;
}

// Block sums of the n per-warp accumulators -> part[i][blockIdx.x] (fixed order); accumulators cleared.
__device__ __forceinline__ void publish(double* acc, int n, double* part) {
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kBlock) {
        double s = 0.0;
        for (int wp = 0; wp < kWarps; ++wp) s += acc[wp * kAcc + i];
        part[(size_t)i * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWarps * kAcc; i += kBlock) acc[i] = 0.0;
}

// After a barrier: tot[i] = sum over blocks of part[i][.] (fixed order; one warp per quantity).
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

// The rows [r0, r1) of this block, two consecutive rows per thread (r0 even): f(i, 2) for a pair, f(i, 1) for a
// single last row.
template <class F>
__device__ __forceinline__ void for_pairs(int r0, int r1, const F& f) {
    for (int i = r0 + 2 * threadIdx.x; i < r1; i += 2 * kBlock) f(i, i + 1 < r1 ? 2 : 1);
}

// The same rows, two row pairs per call (i and i + 2 kBlock) so that the loads of both are in flight together:
// f(i, ci, j, cj) with ci, cj in {0, 1, 2} rows (0: no such pair).
template <class F>
__device__ __forceinline__ void for_pairs2(int r0, int r1, const F& f) {
    for (int i = r0 + 2 * threadIdx.x; i < r1; i += 4 * kBlock) {
        const int j = i + 2 * kBlock;
        f(i, i + 1 < r1 ? 2 : 1, j, j < r1 ? (j + 1 < r1 ? 2 : 1) : 0);
    }
}

__device__ __forceinline__ double2 ld2(const double* p, int n) {
    return n == 2 ? __ldcg(reinterpret_cast<const double2*>(p))
                  : (n == 1 ? make_double2(__ldcg(p), 0.0) : make_double2(0.0, 0.0));
}
__device__ __forceinline__ void st2(double* p, double2 v, int n) {
    if (n == 2)
        *reinterpret_cast<double2*>(p) = v;
    else if (n == 1)
        p[0] = v.x;
}

constexpr int kVb = 3;  // basis vectors per batch of loads (more would spill: 17 warps cap a thread at 96 registers)

// The Gram-Schmidt dots and updates and the update of x run in double-word arithmetic on the FP32 pipes: B300
// retires 2 FP64 FMAs per clock per SM, and with FP64 basis vectors these passes, 2 (j + 1) FMAs per row in
// Arnoldi step j, held the kernel to the FP64 pipe. The basis is stored as float pairs (48 significant bits, no
// conversion when read); each basis term is one compensated product-accumulate (dw::dot_acc, Ogita-Rump-Oishi
// Dot2), whose result is as accurate as an FP64 dot of the same 48-bit inputs. The Arnoldi vector w, the SpMV and
// the Hessenberg arithmetic stay FP64.

// rows i, i + 1 (n of them present) of a double-word vector as one 16-byte load
__device__ __forceinline__ float4 ldw2(const float2* p, int n) {
    if (n == 2) return __ldcg(reinterpret_cast<const float4*>(p));
    if (n == 1) {
        const float2 v = __ldcg(p);
        return make_float4(v.x, v.y, 0.0f, 0.0f);
    }
    return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// acc[warp][i] += (w, v_i) for i < n over the block's rows, and with self (w, w) into acc[warp][n].
__device__ __forceinline__ void dots(const Args& a, double* acc, const double* w, int n, bool self, int r0, int r1) {
    for (int i0 = 0; i0 < n; i0 += kVb) {
        dw::df sum[kVb];
        double ww = 0.0;
#pragma unroll
        for (int t = 0; t < kVb; ++t) sum[t] = dw::make(0.0f);
        const bool with_self = self && i0 == 0;
        for_pairs2(r0, r1, [&](int i, int ci, int j, int cj) {
            const double2 wi = ld2(w + i, ci), wj = ld2(w + j, cj);
            const dw::df w0 = dw::split(wi.x), w1 = dw::split(wi.y), w2 = dw::split(wj.x), w3 = dw::split(wj.y);
            float4 v[kVb], u[kVb];
#pragma unroll
            for (int t = 0; t < kVb; ++t) {
                const float2* vt = a.Vb + (size_t)(i0 + t) * a.ld;
                v[t] = ldw2(vt + i, i0 + t < n ? ci : 0);
                u[t] = ldw2(vt + j, i0 + t < n ? cj : 0);
            }
#pragma unroll
            for (int t = 0; t < kVb; ++t) {
                dw::dot_acc(sum[t], w0, dw::make(v[t].x, v[t].y));
                dw::dot_acc(sum[t], w1, dw::make(v[t].z, v[t].w));
                dw::dot_acc(sum[t], w2, dw::make(u[t].x, u[t].y));
                dw::dot_acc(sum[t], w3, dw::make(u[t].z, u[t].w));
            }
            if (with_self) ww = fma(wj.y, wj.y, fma(wj.x, wj.x, fma(wi.y, wi.y, fma(wi.x, wi.x, ww))));
        });
#pragma unroll
        for (int t = 0; t < kVb; ++t)
            if (i0 + t < n) warp_add(acc, i0 + t, dw::to_double(dw::finish(sum[t])));
        if (with_self) warp_add(acc, n, ww);
    }
}

// w -= sum_{i < n} c_i v_i over the block's rows; with z, also z = dinv w (the next SpMV's input).
__device__ __forceinline__ void subtract(const Args& a, double* w, const double* c_, int n, double* z, int r0, int r1) {
    __shared__ float2 cn[64];  // -c_i as double-word
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += kBlock) dw::store(cn + t, dw::split(-c_[t]));
    __syncthreads();
    for_pairs2(r0, r1, [&](int i, int ci, int j, int cj) {
        const double2 wi = ld2(w + i, ci), wj = ld2(w + j, cj);
        dw::df y0 = dw::split(wi.x), y1 = dw::split(wi.y), y2 = dw::split(wj.x), y3 = dw::split(wj.y);
        for (int i0 = 0; i0 < n; i0 += kVb) {
            float4 v[kVb], u[kVb];
#pragma unroll
            for (int t = 0; t < kVb; ++t) {
                const float2* vt = a.Vb + (size_t)(i0 + t) * a.ld;
                v[t] = ldw2(vt + i, i0 + t < n ? ci : 0);
                u[t] = ldw2(vt + j, i0 + t < n ? cj : 0);
            }
#pragma unroll
            for (int t = 0; t < kVb; ++t) {
                const dw::df ct = i0 + t < n ? dw::load(cn + i0 + t) : dw::make(0.0f);
                dw::dot_acc(y0, ct, dw::make(v[t].x, v[t].y));
                dw::dot_acc(y1, ct, dw::make(v[t].z, v[t].w));
                dw::dot_acc(y2, ct, dw::make(u[t].x, u[t].y));
                dw::dot_acc(y3, ct, dw::make(u[t].z, u[t].w));
            }
        }
        const double2 ni = make_double2(dw::to_double(dw::finish(y0)), dw::to_double(dw::finish(y1)));
        const double2 nj = make_double2(dw::to_double(dw::finish(y2)), dw::to_double(dw::finish(y3)));
        st2(w + i, ni, ci);
        st2(w + j, nj, cj);
        if (z) {
            const double2 di = ld2(a.dinv + i, ci), dj = ld2(a.dinv + j, cj);
            st2(z + i, make_double2(di.x * ni.x, di.y * ni.y), ci);
            st2(z + j, make_double2(dj.x * nj.x, dj.y * nj.y), cj);
        }
    });
}

// r = b - A x at the start of a cycle: w0 = r, z = M^-1 r, partial (r, r)
struct EmStart {
    const Args& a;
    double* v;
    __device__ __forceinline__ double pre(int row) const { return a.b[row]; }
    __device__ __forceinline__ void fin(int row, double ax, double bi) const {
        const double r = bi - ax;
        a.w[0][row] = r;
        a.z[row] = ldcg(a.dinv + row) * r;
        v[0] = fma(r, r, v[0]);
    }
};

// Arnoldi step: w = A M^-1 u / s, v_j = u / s
struct EmArnoldi {
    const double* u;
    double* wn;
    float2* vj;
    double inv;
    __device__ __forceinline__ double pre(int row) const { return ldcg(u + row); }
    __device__ __forceinline__ void fin(int row, double az, double ui) const {
        wn[row] = az * inv;
        dw::store(vj + row, dw::split(ui * inv));
    }
};

template <int L>
__global__ void __launch_bounds__(kBlock, 1) k_gmres(Args a) {
    RAFEM_RING_SETUP(L)
    // columns: 32-bit (L = 1), 16-bit offsets (L = 2) or one pattern per slice (L = 3, values only)
    using Cols = typename std::conditional<
        L == 3, SliceCols, EntryCols<typename std::conditional<L == 2, int16_t, int32_t>::type>>::type;
    Cols sc;
    if constexpr (L == 3)
        sc = SliceCols{a.pat_off, a.pat_pool, a.N};
    else if constexpr (L == 2)
        sc = Cols{a.sc16};
    else
        sc = Cols{a.sc};
    __shared__ double acc[kWarps * kAcc];
    __shared__ double tot[kAcc];
    __shared__ double cs[64], sn[64], g[65], yv[64];
    __shared__ float2 yd[64];  // y as double-word
    __shared__ double sm[kSumMax * kBlock];
    const int m = a.m, N = a.N;
    double* H = a.H + (size_t)blockIdx.x * (m + 1) * m;
    for (int i = threadIdx.x; i < kWarps * kAcc; i += kBlock) acc[i] = 0.0;
    // this block's rows: whole slices [s0, s1); blocks past the last slice own no rows (block-uniform `own`)
    const int S = (N + 31) / 32, spb = (S + gridDim.x - 1) / gridDim.x;
    const int s0 = min((int)blockIdx.x * spb, S), s1 = min(s0 + spb, S);
    const bool own = s0 < s1;
    const int r0 = own ? s0 * 32 : N, r1 = own ? min(s1 * 32, N) : N;
    // partial-sum buffers of consecutive phases are disjoint: S -> PA, O1 -> PB, cycle start and set-up -> PD
    const size_t G = gridDim.x;
    double* PA = a.partial;
    double* PB = PA + (size_t)(m + 2) * G;
    double* PD = PB + (size_t)(m + 2) * G;
    unsigned target = 0;
    bool err = false;
    int iters = 0, status = RAFEM_NOT_CONVERGED, cycles = 0;
    double bb = 0.0, rr = 0.0;
    // dinv = 1 / diag(A); (b, b)
    {
        double v[1] = {0.0};
        for (int row = r0 + threadIdx.x; row < r1; row += kBlock) {
            a.dinv[row] = 1.0 / __ldg(a.A + __ldg(a.diag + row));
            v[0] = fma(a.b[row], a.b[row], v[0]);
        }
        block_sum<1>(v, sm);
        if (threadIdx.x == 0) PD[blockIdx.x] = v[0];
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        totals(PD, 1, tot);
        bb = tot[0];
    }
    const double thr = a.tol * a.tol * (bb > 0.0 ? bb : 1.0);
    // restart length of the current cycle: every solve starts at the full length m
    int m_cur = m;
    double rr_prev = -1.0;
    int stagnant = 0, reorths = 0;
    while (!err) {
        // cycle start: r = b - A x into w[0], z = M^-1 r, (r, r)
        {
            double v[1] = {0.0};
            const bool ok = !own || sell_tile<double, double>(a, ring, a.sp, sc, a.A, a.x, r0, r1, EmStart{a, v});
            block_sum<1>(v, sm);
            if (threadIdx.x == 0) PD[G + blockIdx.x] = v[0];
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) { err = true; break; }
            totals(PD + G, 1, tot);
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
            float2* vj = a.Vb + (size_t)j * a.ld;
            double* Hj = H + (size_t)j * (m + 1);
            // S: w = A M^-1 u / s and v_j = u / s (SpMV through the ring), then h_ij = (w, v_i), i <= j, and (w, w)
            const bool ok = !own || sell_tile<double, double>(a, ring, a.sp, sc, a.A, a.z, r0, r1,
                                                                  EmArnoldi{u, wn, vj, 1.0 / scale});
            dots(a, acc, wn, j + 1, true, r0, r1);
            publish(acc, j + 2, PA);
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) { err = true; break; }
            totals(PA, j + 2, tot);
            double proj = 0.0;  // sum_i h_ij^2 (same order in every block)
            for (int i = 0; i <= j; ++i) proj = fma(tot[i], tot[i], proj);
            const double ww = tot[j + 1];
            double nh2 = ww - proj;
            const bool reorth = !(nh2 >= kReorth * ww);
            if (threadIdx.x == 0)
                for (int i = 0; i <= j; ++i) Hj[i] = tot[i];
            if (reorth) {
                ++reorths;
                // O1: w -= sum_i h_ij v_i, then c_ij = (w, v_i) and (w, w)
                __syncthreads();
                subtract(a, wn, tot, j + 1, nullptr, r0, r1);
                __syncthreads();  // tot is overwritten below; every thread has finished with it
                dots(a, acc, wn, j + 1, true, r0, r1);
                publish(acc, j + 2, PB);
                if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
                totals(PB, j + 2, tot);
                double c2 = 0.0;
                for (int i = 0; i <= j; ++i) c2 = fma(tot[i], tot[i], c2);
                nh2 = tot[j + 1] - c2;
                if (threadIdx.x == 0)
                    for (int i = 0; i <= j; ++i) Hj[i] += tot[i];
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
            // O (or O2): the next basis vector, unnormalised (its norm hn is known), and z = M^-1 of it. tot holds
            // the h_ij of the single pass, or the c_ij of the second pass.
            subtract(a, wn, tot, j + 1, a.z, r0, r1);
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
        for (int i = threadIdx.x; i < k; i += kBlock) dw::store(yd + i, dw::split(yv[i]));
        __syncthreads();
        for_pairs(r0, r1, [&](int i, int c) {
            dw::df t0 = dw::make(0.0f), t1 = dw::make(0.0f);
            for (int i0 = 0; i0 < k; i0 += kVb) {
                float4 v[kVb];
#pragma unroll
                for (int q = 0; q < kVb; ++q) v[q] = ldw2(a.Vb + (size_t)(i0 + q) * a.ld + i, i0 + q < k ? c : 0);
#pragma unroll
                for (int q = 0; q < kVb; ++q) {
                    const dw::df yq = i0 + q < k ? dw::load(yd + i0 + q) : dw::make(0.0f);
                    dw::dot_acc(t0, yq, dw::make(v[q].x, v[q].y));
                    dw::dot_acc(t1, yq, dw::make(v[q].z, v[q].w));
                }
            }
            const double tx = dw::to_double(dw::finish(t0)), ty = dw::to_double(dw::finish(t1));
            // x is the caller's buffer (no alignment beyond 8 bytes is assumed): scalar accesses
            const double2 d = ld2(a.dinv + i, c);
            a.x[i] = fma(d.x, tx, a.x[i]);
            if (c == 2) a.x[i + 1] = fma(d.y, ty, a.x[i + 1]);
        });
        if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
    }
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

void* kernel_for(const GmresArgs& s) {
    return s.pat_off ? (void*)k_gmres<3> : (s.sc16 ? (void*)k_gmres<2> : (void*)k_gmres<1>);
}

}  // namespace

int gmres_max_blocks(int /*m*/) {
    int dev = 0, sms = 0, per1 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    int per = 1;
    for (void* k : {(void*)k_gmres<1>, (void*)k_gmres<2>, (void*)k_gmres<3>}) {
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k, kBlock, kRingBytes) != cudaSuccess) return 0;
        per = per1 < per ? per1 : per;
    }
    return sms * (per < 1 ? per : 1);
}

int gmres_partial_slots(int m) { return 2 * (m + 2) + 2; }

cudaError_t launch_gmres(const GmresArgs& s, int grid, cudaStream_t st) {
    Args a{s.N, s.m, s.m_min, s.ld, s.sp, s.sc, s.sc16, s.pat_off, s.pat_pool, s.A, s.diag, s.b, s.x, reinterpret_cast<float2*>(s.V), {s.w0, s.w1}, s.z, s.dinv, s.H,
           s.partial, s.bar, s.inst, s.tol, s.max_iter, s.spin_limit_ns};
    cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    if (s.bar_missing > 0 && (e = launch_barrier_reset(s.bar, s.bar_missing, st)) != cudaSuccess) return e;
    void* params[] = {&a};
    return cudaLaunchCooperativeKernel(kernel_for(s), dim3(grid), dim3(kBlock), params, kRingBytes, st);
}

}  // namespace rafem
