// Persistent Jacobi-preconditioned BiCGSTAB (FP64) for general (nonsymmetric) systems on the SELL-32 layout, for
// scalar rows (B = 1) or 2 x 2 block rows (B = 2: the monolithic potential/temperature system, block Jacobi).
//
// Sec. II-B: CG suits symmetric positive-definite systems; for nonsymmetric ones a method that does not need
// symmetry is used (the paper's own choice there is GMRES). BiCGSTAB (van der Vorst) with right
// preconditioning M = diag(A) runs here as one cooperative launch:
//   A (row-local):  p = r + beta (p - omega v),  ph = M^-1 p                         -- barrier --
//   B (SpMV):       v = A ph,  partial (rh, v)                                       -- barrier: alpha --
//   C (row-local):  s = r - alpha v,  sh = M^-1 s,  partial (s, s)                   -- barrier --
//   D (SpMV):       t = A sh,  partials (t, s), (t, t)                               -- barrier: omega --
//   E (row-local):  x += alpha ph + omega sh,  r = s - omega t,  partials (r, r), (rh, r)  -- barrier: rho, beta --
// with the shadow residual rh = r_0. Every block reduces the per-block partial sums itself in a fixed order
// (deterministic); consecutive phases use disjoint partial-sum slots. Breakdown ((rh, v) = 0, rho = 0,
// (t, t) = 0) stops the solve with RAFEM_ERR_BREAKDOWN. Every barrier wait is bounded.
#include <cuda_runtime.h>

#include <cmath>

#include "grid_sync.cuh"
#include "internal.h"

namespace rafem {

namespace {

constexpr int kBlock = 512;
constexpr int kWarps = kBlock / 32;
constexpr int kBatch = 8;
constexpr int kSlots = 6;

struct Args {
    int N;                // block rows
    const int32_t* sp;
    const int32_t* sc;
    const int16_t* sc16;
    const double* A;      // B x B block per stored entry (row-major within the block)
    const int32_t* diag;
    const double* b;
    double* x;
    double *r, *rh, *p, *ph, *v, *s, *sh, *t, *dinv;  // B values per row (dinv: B x B)
    double* partial;
    GridBarrier* bar;
    InstState* inst;
    double tol;
    int max_iter;
    long long spin_limit_ns;
    double* newton;       // inexact Newton: ||R||^2 of the previous linear solve of this step (0: the first), or null
};

// Forcing terms of the inexact Newton iteration of the monolithic step (Eisenstat and Walker, "Choosing the forcing
// terms in an inexact Newton method", SIAM J. Sci. Comput. 17 (1996), their second choice): the linear solve of
// Newton iteration k stops at ||r|| <= eta_k ||R_k|| with eta_k = gamma (||R_k|| / ||R_{k-1}||)^alpha, gamma = 0.9,
// alpha = 2, kept within [tol, kEtaMax]; the first iteration of a step uses kEta0.
constexpr double kEtaGamma = 0.9;
constexpr double kEta0 = 1e-3;
constexpr double kEtaMax = 1e-2;

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ double* slot(const Args& a, int k) { return a.partial + (size_t)k * gridDim.x; }

// slice s always belongs to warp (s mod total warps)
template <class Fn>
__device__ __forceinline__ void for_slices(int S, const Fn& f) {
    const int tw = gridDim.x * kWarps;
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * kWarps + (threadIdx.x >> 5); s < S; s += tw) f(s, s * 32 + lane);
}

template <int NQ>
__device__ __forceinline__ void publish(const double (&v)[NQ], double* sm, double* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q * kBlock + threadIdx.x] = v[q];
    __syncthreads();
    if (warp < NQ) {
        double acc = sm[warp * kBlock + lane];
#pragma unroll
        for (int k = 1; k < kWarps; ++k) acc += sm[warp * kBlock + 32 * k + lane];
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[(size_t)warp * gridDim.x + blockIdx.x] = acc;
    }
}

template <int NQ>
__device__ __forceinline__ void totals(const double* part, double* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < NQ) {
        double acc = 0.0;
        for (int t = lane; t < (int)gridDim.x; t += 32) acc += ldcg(part + (size_t)warp * gridDim.x + t);
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_tot[warp] = acc;
    }
    __syncthreads();
}

// (A y)_row (B values) over the SELL-32 slice s; entries are loaded in batches before the gathers that depend on
// them
template <int B>
__device__ __forceinline__ void spmv_row(const Args& a, const double* y, int s, int row, double (&out)[B]) {
    const int lane = row & 31;
    const int base = __ldg(a.sp + s), w = (__ldg(a.sp + s + 1) - base) >> 5;
#pragma unroll
    for (int q = 0; q < B; ++q) out[q] = 0.0;
    for (int k = 0; k < w; k += kBatch) {
        int c[kBatch];
        double m[kBatch][B * B], yv[kBatch][B];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            const int pos = base + 32 * (k + t) + lane;
            const bool ok = k + t < w;
            c[t] = ok ? (a.sc16 ? row + (int)__ldg(a.sc16 + pos) : __ldg(a.sc + pos)) : -1;
#pragma unroll
            for (int q = 0; q < B * B; ++q) m[t][q] = ok ? __ldg(a.A + (size_t)B * B * pos + q) : 0.0;
        }
#pragma unroll
        for (int t = 0; t < kBatch; ++t)
#pragma unroll
            for (int q = 0; q < B; ++q) yv[t][q] = c[t] >= 0 ? ldcg(y + (size_t)B * c[t] + q) : 0.0;
#pragma unroll
        for (int t = 0; t < kBatch; ++t)
#pragma unroll
            for (int i = 0; i < B; ++i)
#pragma unroll
                for (int q = 0; q < B; ++q) out[i] = fma(m[t][B * i + q], yv[t][q], out[i]);
    }
}

// z = D^-1 u with the inverse diagonal block of the row
template <int B>
__device__ __forceinline__ void apply_dinv(const double* dinv, int row, const double (&u)[B], double (&z)[B]) {
#pragma unroll
    for (int i = 0; i < B; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < B; ++q) acc = fma(dinv[(size_t)B * B * row + B * i + q], u[q], acc);
        z[i] = acc;
    }
}

template <int B>
__global__ void __launch_bounds__(kBlock, 1) k_bicgstab(Args a) {
    __shared__ double sm[2 * kBlock];
    __shared__ double s_tot[2];
    const int N = a.N, S = (N + 31) / 32;
    unsigned target = 0;
    bool err = false;
    int iters = 0, status = RAFEM_NOT_CONVERGED;
    double bb, rr, rho, alpha = 1.0, omega = 1.0, beta = 0.0;
    // r = b - A x, rh = r, p = v = 0, inverse diagonal blocks; (b, b), (r, r)
    {
        double q[2] = {0.0, 0.0};
        for_slices(S, [&](int s, int row) {
            if (row >= N) return;
            double ax[B];
            spmv_row<B>(a, a.x, s, row, ax);
            const double* d = a.A + (size_t)B * B * __ldg(a.diag + row);
            if constexpr (B == 1) {
                a.dinv[row] = 1.0 / __ldg(d);
            } else {
                const double d00 = __ldg(d), d01 = __ldg(d + 1), d10 = __ldg(d + 2), d11 = __ldg(d + 3);
                const double inv = 1.0 / (d00 * d11 - d01 * d10);
                double* o = a.dinv + 4 * (size_t)row;
                o[0] = d11 * inv;
                o[1] = -d01 * inv;
                o[2] = -d10 * inv;
                o[3] = d00 * inv;
            }
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const size_t i = (size_t)B * row + k;
                const double bi = a.b[i], ri = bi - ax[k];
                a.r[i] = ri;
                a.rh[i] = ri;
                a.p[i] = 0.0;
                a.v[i] = 0.0;
                q[0] = fma(bi, bi, q[0]);
                q[1] = fma(ri, ri, q[1]);
            }
        });
        publish<2>(q, sm, slot(a, 4));
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        totals<2>(slot(a, 4), s_tot);
        bb = s_tot[0];
        rr = s_tot[1];
        rho = rr;  // (rh, r) with rh = r
    }
    double tol = a.tol;
    if (a.newton) {
        const double prev = *(volatile double*)a.newton;
        const double eta = prev > 0.0 ? kEtaGamma * (bb / prev) : kEta0;  // (||R_k|| / ||R_{k-1}||)^2 = bb / prev
        tol = fmin(fmax(eta, a.tol), kEtaMax);
    }
    const double thr = tol * tol * (bb > 0.0 ? bb : 1.0);
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
        for_slices(S, [&](int, int row) {
            if (row >= N) return;
            double pv[B], z[B];
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const size_t i = (size_t)B * row + k;
                pv[k] = fma(beta, fma(-omega, a.v[i], a.p[i]), a.r[i]);
                a.p[i] = pv[k];
            }
            apply_dinv<B>(a.dinv, row, pv, z);
#pragma unroll
            for (int k = 0; k < B; ++k) a.ph[(size_t)B * row + k] = z[k];
        });
        if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
        // B: v = A ph, (rh, v)
        {
            double q[1] = {0.0};
            for_slices(S, [&](int s, int row) {
                if (row >= N) return;
                double vv[B];
                spmv_row<B>(a, a.ph, s, row, vv);
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const size_t i = (size_t)B * row + k;
                    a.v[i] = vv[k];
                    q[0] = fma(a.rh[i], vv[k], q[0]);
                }
            });
            publish<1>(q, sm, slot(a, 0));
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<1>(slot(a, 0), s_tot);
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
            for_slices(S, [&](int, int row) {
                if (row >= N) return;
                double sv[B], z[B];
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const size_t i = (size_t)B * row + k;
                    sv[k] = fma(-alpha, a.v[i], a.r[i]);
                    a.s[i] = sv[k];
                    q[0] = fma(sv[k], sv[k], q[0]);
                }
                apply_dinv<B>(a.dinv, row, sv, z);
#pragma unroll
                for (int k = 0; k < B; ++k) a.sh[(size_t)B * row + k] = z[k];
            });
            publish<1>(q, sm, slot(a, 1));
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<1>(slot(a, 1), s_tot);
            if (s_tot[0] <= thr) {  // converged on the half step: x += alpha ph
                for_slices(S, [&](int, int row) {
                    if (row >= N) return;
#pragma unroll
                    for (int k = 0; k < B; ++k) {
                        const size_t i = (size_t)B * row + k;
                        a.x[i] = fma(alpha, a.ph[i], a.x[i]);
                    }
                });
                ++iters;
                status = RAFEM_OK;
                break;
            }
        }
        // D: t = A sh, (t, s), (t, t)
        {
            double q[2] = {0.0, 0.0};
            for_slices(S, [&](int s, int row) {
                if (row >= N) return;
                double tv[B];
                spmv_row<B>(a, a.sh, s, row, tv);
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const size_t i = (size_t)B * row + k;
                    a.t[i] = tv[k];
                    q[0] = fma(tv[k], a.s[i], q[0]);
                    q[1] = fma(tv[k], tv[k], q[1]);
                }
            });
            publish<2>(q, sm, slot(a, 2));
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<2>(slot(a, 2), s_tot);
            if (!(s_tot[1] > 0.0)) {
                status = s_tot[1] == s_tot[1] ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
                break;
            }
            omega = s_tot[0] / s_tot[1];
        }
        // E: x += alpha ph + omega sh, r = s - omega t, (r, r), (rh, r)
        {
            double q[2] = {0.0, 0.0};
            for_slices(S, [&](int, int row) {
                if (row >= N) return;
#pragma unroll
                for (int k = 0; k < B; ++k) {
                    const size_t i = (size_t)B * row + k;
                    a.x[i] = fma(omega, a.sh[i], fma(alpha, a.ph[i], a.x[i]));
                    const double ri = fma(-omega, a.t[i], a.s[i]);
                    a.r[i] = ri;
                    q[0] = fma(ri, ri, q[0]);
                    q[1] = fma(a.rh[i], ri, q[1]);
                }
            });
            publish<2>(q, sm, slot(a, 4));
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<2>(slot(a, 4), s_tot);
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
    // true residual
    double relres = 0.0;
    if (!err && !grid_barrier(a.bar, a.spin_limit_ns, target)) {
        double q[1] = {0.0};
        for_slices(S, [&](int s, int row) {
            if (row >= N) return;
            double ax[B];
            spmv_row<B>(a, a.x, s, row, ax);
#pragma unroll
            for (int k = 0; k < B; ++k) {
                const double ri = a.b[(size_t)B * row + k] - ax[k];
                q[0] = fma(ri, ri, q[0]);
            }
        });
        publish<1>(q, sm, slot(a, 3));
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        totals<1>(slot(a, 3), s_tot);
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
        if (a.newton) *a.newton = bb;
    }
}

}  // namespace

int bicgstab_max_blocks(int block) {
    if (block == 1) return bicgstab_ring_max_blocks();
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const void* f = (const void*)k_bicgstab<2>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, kBlock, 0) != cudaSuccess) return 0;
    return sms * (per < 1 ? per : 1);
}

int bicgstab_partial_slots() { return kSlots > bicgstab_ring_partial_slots() ? kSlots : bicgstab_ring_partial_slots(); }

cudaError_t launch_bicgstab(const BicgArgs& s, int grid, cudaStream_t st) {
    if (s.block == 1) return launch_bicgstab_ring(s, grid, st);
    Args a{s.N, s.sp, s.sc, s.sc16, s.A, s.diag, s.b, s.x, s.r, s.rh, s.p, s.ph, s.v, s.s, s.sh, s.t, s.dinv,
           s.partial, s.bar, s.inst, s.tol, s.max_iter, s.spin_limit_ns, s.newton};
    cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    if (s.bar_missing > 0 && (e = launch_barrier_reset(s.bar, s.bar_missing, st)) != cudaSuccess) return e;
    void* params[] = {&a};
    const void* f = (const void*)k_bicgstab<2>;
    return cudaLaunchCooperativeKernel(f, dim3(grid), dim3(kBlock), params, 0, st);
}

}  // namespace rafem
