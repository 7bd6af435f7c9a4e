// Persistent Jacobi-preconditioned BiCGSTAB (FP64) for scalar nonsymmetric systems, with both SpMVs of an iteration
// streaming the matrix through the shared-memory ring of the CG kernels (sell_ring.cuh). Sec. II-B: for systems
// that are not symmetric positive definite a method that does not need symmetry is used. BiCGSTAB (van der Vorst)
// with right preconditioning M = diag(A), one cooperative launch per solve, five grid barriers per iteration:
//   A (row-local):  p = r + beta (p - omega v),  ph = M^-1 p                         -- barrier --
//   B (SpMV):       v = A ph,  partial (rh, v)                                       -- barrier: alpha --
//   C (row-local):  s = r - alpha v,  sh = M^-1 s,  partial (s, s)                   -- barrier --
//   D (SpMV):       t = A sh,  partials (t, s), (t, t)                               -- barrier: omega --
//   E (row-local):  x += alpha ph + omega sh,  r = s - omega t,  partials (r, r), (rh, r)  -- barrier: rho, beta --
// with the shadow residual rh = r_0. Block b owns the b-th run of slices in every phase, so the row-local phases
// touch only the block's own rows (two consecutive rows per thread, 16-byte accesses). Every block reduces the
// per-block sums itself in a fixed order (deterministic); consecutive reductions use distinct slots. Breakdown
// ((rh, v) = 0, rho = 0, (t, t) = 0) stops the solve with RAFEM_ERR_BREAKDOWN; every wait is bounded. The 2 x 2
// block form of the monolithic step keeps the kernel of bicgstab.cu.
#include <cuda_runtime.h>

#include <cmath>

#include "grid_sync.cuh"
#include "internal.h"
#include "sell_ring.cuh"

namespace rafem {

namespace {

using namespace sell;

enum { S_RV = 0, S_SS = 1, S_TS = 2, S_TT = 3, S_RR = 4, S_RHR = 5, S_TRUE = 6, S_COUNT = 7 };

struct Args {
    int N;
    const int32_t* sp;
    const int32_t* sc;
    const int16_t* sc16;
    const int32_t* pat_off;
    const int32_t* pat_pool;
    const double* A;
    const int32_t* diag;
    const double* b;
    double* x;
    double *r, *rh, *p, *ph, *v, *s, *sh, *t, *dinv;
    double* partial;  // [S_COUNT][grid]
    GridBarrier* bar;
    InstState* inst;
    double tol;
    int max_iter;
    long long spin_limit_ns;
};

template <int L, class Emit>
__device__ __forceinline__ bool spmv(const Args& a, Ring& g, const double* xin, int r0, int r1, const Emit& em) {
    if (r0 >= r1) return __syncthreads_and(1);
    if constexpr (L == 1)
        return sell_tile<double, double>(a, g, a.sp, EntryCols<int32_t>{a.sc}, a.A, xin, r0, r1, em);
    else if constexpr (L == 2)
        return sell_tile<double, double>(a, g, a.sp, EntryCols<int16_t>{a.sc16}, a.A, xin, r0, r1, em);
    else
        return sell_tile<double, double>(a, g, a.sp, SliceCols{a.pat_off, a.pat_pool, a.N}, a.A, xin, r0, r1, em);
}

// Rows [r0, r1) of this block, two consecutive rows per thread (r0 even): f(i, n) with n = 2 or 1 rows.
template <class F>
__device__ __forceinline__ void for_pairs(int r0, int r1, const F& f) {
    for (int i = r0 + 2 * threadIdx.x; i < r1; i += 2 * kBlock) f(i, i + 1 < r1 ? 2 : 1);
}
__device__ __forceinline__ double2 ld2(const double* p, int n) {
    return n == 2 ? __ldcg(reinterpret_cast<const double2*>(p)) : make_double2(__ldcg(p), 0.0);
}
__device__ __forceinline__ void st2(double* p, double2 v, int n) {
    if (n == 2)
        *reinterpret_cast<double2*>(p) = v;
    else
        p[0] = v.x;
}

template <int NQ>
__device__ __forceinline__ void publish(double (&v)[NQ], double* sm, double* part, int slot0) {
    block_sum<NQ>(v, sm);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) part[(size_t)(slot0 + q) * gridDim.x + blockIdx.x] = v[q];
}
template <int NQ>
__device__ __forceinline__ void totals(const double* part, int slot0, double* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < NQ) {
        double acc = 0.0;
        for (int t = lane; t < (int)gridDim.x; t += 32) acc += __ldcg(part + (size_t)(slot0 + warp) * gridDim.x + t);
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_tot[warp] = acc;
    }
    __syncthreads();
}

// r = b - A x, rh = r, p = v = 0, dinv = 1 / a_ii; (b, b), (r, r)
struct EmInit {
    const Args& a;
    double* q;
    __device__ __forceinline__ double pre(int row) const { return a.b[row]; }
    __device__ __forceinline__ void fin(int row, double ax, double bi) const {
        const double ri = bi - ax;
        a.r[row] = ri;
        a.rh[row] = ri;
        a.p[row] = 0.0;
        a.v[row] = 0.0;
        a.dinv[row] = 1.0 / __ldg(a.A + __ldg(a.diag + row));
        q[0] = fma(bi, bi, q[0]);
        q[1] = fma(ri, ri, q[1]);
    }
};
// v = A ph; (rh, v)
struct EmV {
    const Args& a;
    double* q;
    __device__ __forceinline__ double pre(int row) const { return ldcg(a.rh + row); }
    __device__ __forceinline__ void fin(int row, double av, double rhi) const {
        a.v[row] = av;
        q[0] = fma(rhi, av, q[0]);
    }
};
// t = A sh; (t, s), (t, t)
struct EmT {
    const Args& a;
    double* q;
    __device__ __forceinline__ double pre(int row) const { return ldcg(a.s + row); }
    __device__ __forceinline__ void fin(int row, double at, double si) const {
        a.t[row] = at;
        q[0] = fma(at, si, q[0]);
        q[1] = fma(at, at, q[1]);
    }
};
// (b - A x, b - A x)
struct EmTrue {
    const double* b;
    double* q;
    __device__ __forceinline__ double pre(int row) const { return b[row]; }
    __device__ __forceinline__ void fin(int, double ax, double bi) const {
        const double ri = bi - ax;
        q[0] = fma(ri, ri, q[0]);
    }
};

template <int L>
__global__ void __launch_bounds__(kBlock, 1) k_bicgstab_ring(Args a) {
    RAFEM_RING_SETUP(L)
    __shared__ double sm[kSumMax * kBlock];
    __shared__ double s_tot[2];
    const int N = a.N;
    const int S = (N + 31) / 32, spb = (S + gridDim.x - 1) / gridDim.x;
    const int s0 = min((int)blockIdx.x * spb, S), s1 = min(s0 + spb, S);
    const int r0 = s0 < s1 ? 32 * s0 : N, r1 = s0 < s1 ? min(32 * s1, N) : N;
    unsigned target = 0;
    bool err = false, ok = true;
    int iters = 0, status = RAFEM_NOT_CONVERGED;
    double bb, rr, rho, alpha = 1.0, omega = 1.0, beta;
    {
        double q[2] = {0.0, 0.0};
        ok = spmv<L>(a, ring, a.x, r0, r1, EmInit{a, q});
        publish<2>(q, sm, a.partial, S_RR);
        err = grid_barrier(a.bar, a.spin_limit_ns, target) || !ok;
        totals<2>(a.partial, S_RR, s_tot);
        bb = s_tot[0];
        rr = s_tot[1];
        rho = rr;  // (rh, r) with rh = r
    }
    const double thr = a.tol * a.tol * (bb > 0.0 ? bb : 1.0);
    bool done = err || !(rr > thr);
    if (!err && !(rr == rr)) status = RAFEM_ERR_NONFINITE;
    else if (done) status = RAFEM_OK;
    double rho_prev = 1.0;
    while (!done && !err) {
        if (!(rho != 0.0) || !(omega != 0.0)) {
            status = rho == rho ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
            break;
        }
        beta = (rho / rho_prev) * (alpha / omega);
        // A: p = r + beta (p - omega v), ph = M^-1 p
        for_pairs(r0, r1, [&](int i, int n) {
            const double2 ri = ld2(a.r + i, n), pi = ld2(a.p + i, n), vi = ld2(a.v + i, n), di = ld2(a.dinv + i, n);
            const double2 pn = make_double2(fma(beta, fma(-omega, vi.x, pi.x), ri.x),
                                            fma(beta, fma(-omega, vi.y, pi.y), ri.y));
            st2(a.p + i, pn, n);
            st2(a.ph + i, make_double2(di.x * pn.x, di.y * pn.y), n);
        });
        if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
        // B: v = A ph, (rh, v)
        {
            double q[1] = {0.0};
            ok = spmv<L>(a, ring, a.ph, r0, r1, EmV{a, q});
            publish<1>(q, sm, a.partial, S_RV);
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) { err = true; break; }
            totals<1>(a.partial, S_RV, s_tot);
            const double rv = s_tot[0];
            if (!(rv != 0.0)) {
                status = rv == rv ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
                break;
            }
            alpha = rho / rv;
        }
        // C: s = r - alpha v, sh = M^-1 s, (s, s)
        {
            double q[1] = {0.0};
            for_pairs(r0, r1, [&](int i, int n) {
                const double2 ri = ld2(a.r + i, n), vi = ld2(a.v + i, n), di = ld2(a.dinv + i, n);
                const double2 si = make_double2(fma(-alpha, vi.x, ri.x), fma(-alpha, vi.y, ri.y));
                st2(a.s + i, si, n);
                st2(a.sh + i, make_double2(di.x * si.x, di.y * si.y), n);
                q[0] = fma(si.y, si.y, fma(si.x, si.x, q[0]));
            });
            publish<1>(q, sm, a.partial, S_SS);
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<1>(a.partial, S_SS, s_tot);
            if (s_tot[0] <= thr) {  // converged on the half step: x += alpha ph
                for_pairs(r0, r1, [&](int i, int n) {
                    const double2 hi = ld2(a.ph + i, n);
                    a.x[i] = fma(alpha, hi.x, a.x[i]);  // the caller's buffer: scalar accesses
                    if (n == 2) a.x[i + 1] = fma(alpha, hi.y, a.x[i + 1]);
                });
                ++iters;
                status = RAFEM_OK;
                break;
            }
        }
        // D: t = A sh, (t, s), (t, t)
        {
            double q[2] = {0.0, 0.0};
            ok = spmv<L>(a, ring, a.sh, r0, r1, EmT{a, q});
            publish<2>(q, sm, a.partial, S_TS);
            if (grid_barrier(a.bar, a.spin_limit_ns, target) || !ok) { err = true; break; }
            totals<2>(a.partial, S_TS, s_tot);
            if (!(s_tot[1] > 0.0)) {
                status = s_tot[1] == s_tot[1] ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
                break;
            }
            omega = s_tot[0] / s_tot[1];
        }
        // E: x += alpha ph + omega sh, r = s - omega t, (r, r), (rh, r)
        {
            double q[2] = {0.0, 0.0};
            for_pairs(r0, r1, [&](int i, int n) {
                const double2 hi = ld2(a.ph + i, n), shi = ld2(a.sh + i, n), si = ld2(a.s + i, n),
                              ti = ld2(a.t + i, n), rhi = ld2(a.rh + i, n);
                // x is the caller's buffer (8-byte alignment only): scalar accesses
                a.x[i] = fma(omega, shi.x, fma(alpha, hi.x, a.x[i]));
                if (n == 2) a.x[i + 1] = fma(omega, shi.y, fma(alpha, hi.y, a.x[i + 1]));
                const double2 rn = make_double2(fma(-omega, ti.x, si.x), fma(-omega, ti.y, si.y));
                st2(a.r + i, rn, n);
                q[0] = fma(rn.y, rn.y, fma(rn.x, rn.x, q[0]));
                q[1] = fma(rhi.y, rn.y, fma(rhi.x, rn.x, q[1]));
            });
            publish<2>(q, sm, a.partial, S_RR);
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<2>(a.partial, S_RR, s_tot);
            rr = s_tot[0];
            rho_prev = rho;
            rho = s_tot[1];
            ++iters;
            if (!(rr == rr)) {
                status = RAFEM_ERR_NONFINITE;
                break;
            }
            if (rr <= thr) {
                status = RAFEM_OK;
                break;
            }
            if (iters >= a.max_iter) break;
        }
    }
    // true residual of the final x (x of other blocks is gathered: a barrier first)
    double relres = 0.0;
    if (!err && !grid_barrier(a.bar, a.spin_limit_ns, target)) {
        double q[1] = {0.0};
        ok = spmv<L>(a, ring, a.x, r0, r1, EmTrue{a.b, q});
        publish<1>(q, sm, a.partial, S_TRUE);
        err = grid_barrier(a.bar, a.spin_limit_ns, target) || !ok;
        totals<1>(a.partial, S_TRUE, s_tot);
        relres = sqrt(s_tot[0] / (bb > 0.0 ? bb : 1.0));
    } else {
        err = true;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        InstState st = {};
        st.bb = bb;
        st.rr = rr;
        st.iters = iters;
        st.status = err ? (a.bar->err ? a.bar->err : RAFEM_ERR_TIMEOUT) : status;
        st.relres = relres;
        a.inst[0] = st;
    }
}

void* kernel_for(int L) {
    return L == 3 ? (void*)k_bicgstab_ring<3> : (L == 2 ? (void*)k_bicgstab_ring<2> : (void*)k_bicgstab_ring<1>);
}

}  // namespace

int bicgstab_ring_max_blocks() {
    int dev = 0, sms = 0, per = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    for (int L = 1; L <= 3; ++L) {
        int q = 0;
        if (cudaFuncSetAttribute(kernel_for(L), cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes) != cudaSuccess)
            return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q, kernel_for(L), kBlock, kRingBytes) != cudaSuccess) return 0;
        per = q < per ? q : per;
    }
    return sms * per;
}

int bicgstab_ring_partial_slots() { return S_COUNT; }

cudaError_t launch_bicgstab_ring(const BicgArgs& s, int grid, cudaStream_t st) {
    Args a{s.N, s.sp, s.sc, s.sc16, s.pat_off, s.pat_pool, s.A, s.diag, s.b, s.x, s.r, s.rh, s.p, s.ph, s.v, s.s,
           s.sh, s.t, s.dinv, s.partial, s.bar, s.inst, s.tol, s.max_iter, s.spin_limit_ns};
    cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    if (s.bar_missing > 0 && (e = launch_barrier_reset(s.bar, s.bar_missing, st)) != cudaSuccess) return e;
    const int L = s.pat_off ? 3 : (s.sc16 ? 2 : 1);
    void* params[] = {&a};
    return cudaLaunchCooperativeKernel(kernel_for(L), dim3(grid), dim3(kBlock), params, kRingBytes, st);
}

}  // namespace rafem
