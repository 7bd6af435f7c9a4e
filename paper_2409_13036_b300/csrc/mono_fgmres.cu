// Newton linear solve of the monolithic step (the 2N x 2N coupled system of Table II) by flexible GMRES, right-
// preconditioned by one block Gauss-Seidel sweep over the (V, T) blocks whose diagonal-block solves are loose
// Jacobi-PCG solves of the split systems:
//   z_V = A_V^-1 r_V   (persistent CG on the assembled potential matrix, relative residual 0.4, from zero)
//   z_T = A_T^-1 (r_T - J_TV z_V)
// A_V (sigma at T^n, from the staggered start of the step) and A_T (constant) stand in for the Jacobian's
// diagonal blocks, which differ from them only by the step's own temperature change and the Joule term's
// derivative in T. The preconditioner varies from one application to the next (the inner solves stop on a
// residual test), hence the flexible form (Saad, "A flexible inner-outer preconditioned GMRES algorithm", SIAM J.
// Sci. Comput. 14(2), 1993): the preconditioned vectors z_j are kept and the correction is sum_j y_j z_j. Each outer
// iteration is a fixed sequence of launches; once the state's done flag is set (converged to the Newton forcing
// term, out of iterations, or broken down) every later kernel and inner solve returns at once, so the sequence can
// sit in the step's captured graph without a conditional node. Gram-Schmidt is classical, with a second pass only
// when the first keeps less than 1% of (w, w), the norm from the Pythagorean identity of the last pass. Reductions
// are two-pass and in a fixed order: repeated runs give the same bits.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace rafem {

namespace {

constexpr int kThreads = 256;
constexpr int kDots = kFgMax + 2;  // at most kFgMax + 1 basis vectors and (w, w)

inline int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

// Forcing terms of the inexact Newton iteration (Eisenstat and Walker, "Choosing the forcing terms in an inexact
// Newton method", SIAM J. Sci. Comput. 17(1), 1996, choice 2 with gamma = 0.9, alpha = 2), within
// [max(tol, kEtaMin), kEtaMax]; the first Newton iteration of a step uses kEta0. The floor kEtaMin: once the
// Newton iteration converges quadratically, choice 2 asks for reductions far below what the step's stopping test
// (max |dT| < corrector_tol) needs, and each further decade costs outer iterations while another Newton
// iteration (a new residual from the exact assembly) costs one assembly.
constexpr double kEtaGamma = 0.9;
constexpr double kEta0 = 1e-3;
constexpr double kEtaMin = 1e-6;
constexpr double kEtaMax = 1e-2;

__device__ __forceinline__ bool skipped(const FgState* st) { return *(volatile const int*)&st->done != 0; }

// partial[q][block] = sum over the block's entries of w * V_q (q < nv) and w * w (q = nv); fixed order
__global__ void __launch_bounds__(kThreads) k_fg_dots(int n2, const double* __restrict__ w,
                                                      const double* __restrict__ V, size_t ld, int nv,
                                                      const FgState* st, double* __restrict__ partial, int pass) {
    if (skipped(st) || (pass == 2 && st->single)) return;
    __shared__ double sm[kDots][kThreads / 32];
    double acc[kDots];
#pragma unroll
    for (int q = 0; q < kDots; ++q) acc[q] = 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n2; i += gridDim.x * kThreads) {
        const double wi = w[i];
#pragma unroll
        for (int q = 0; q < kDots - 1; ++q)
            if (q < nv) acc[q] = fma(wi, V[q * ld + i], acc[q]);
        acc[kDots - 1] = fma(wi, wi, acc[kDots - 1]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kDots; ++q) {
        double v = acc[q];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm[q][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDots) {
        const int q = threadIdx.x;
        double v = 0.0;
        for (int k = 0; k < kThreads / 32; ++k) v += sm[q][k];
        // the self product goes to slot nv, right after the basis products
        const int slot = q == kDots - 1 ? nv : q;
        if (q < nv || q == kDots - 1) partial[(size_t)slot * gridDim.x + blockIdx.x] = v;
    }
}

// start of a Newton linear solve: beta = ||R|| (partial slot 0 of a dots launch with nv = 0), forcing term, state
__global__ void k_fg_init(FgState* st, const double* partial, int G, double* newton_rr, double tol) {
    // one warp: lanes take every 32nd block partial, then a fixed shuffle tree
    double v = 0.0;
    for (int b = threadIdx.x; b < G; b += 32) v += partial[b];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x != 0) return;
    const double bb = v;
    const double prev = *newton_rr;
    const double eta = prev > 0.0 ? kEtaGamma * (bb / prev) : kEta0;  // (||R_k|| / ||R_{k-1}||)^2 = bb / prev
    *newton_rr = bb;
    FgState s{};
    s.beta = sqrt(bb);
    s.eta = fmin(fmax(eta, fmax(tol, kEtaMin)), kEtaMax);
    s.g[0] = s.beta;
    s.scale = s.beta > 0.0 ? 1.0 / s.beta : 0.0;
    s.status = RAFEM_OK;
    if (!isfinite(bb)) s.status = RAFEM_ERR_NONFINITE;
    s.done = !(s.beta > 0.0) || !isfinite(bb);
    *st = s;
}

__global__ void __launch_bounds__(kThreads) k_fg_scale(int n2, const double* __restrict__ src, double* __restrict__ dst,
                                                       const FgState* st) {
    if (skipped(st)) return;
    const double sc = st->scale;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n2; i += gridDim.x * kThreads) dst[i] = src[i] * sc;
}

// preconditioner input: the V and T parts of v, and zero initial guesses for the two inner solves
__global__ void __launch_bounds__(kThreads) k_fg_split(int N, const double* __restrict__ v, double* __restrict__ rV,
                                                       double* __restrict__ rT, double* __restrict__ zV,
                                                       double* __restrict__ zT, const FgState* st) {
    if (skipped(st)) return;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < N; i += gridDim.x * kThreads) {
        const double2 p = reinterpret_cast<const double2*>(v)[i];
        rV[i] = p.x;
        rT[i] = p.y;
        zV[i] = 0.0;
        zT[i] = 0.0;
    }
}

// inner solve statistics (a skipped solve left the reset state: no iterations, status OK)
__global__ void k_fg_count(FgState* st, const InstState* inst, int which) {
    const InstState s = inst[0];
    if (which == RAFEM_SYS_V)
        st->itV += s.iters;
    else
        st->itT += s.iters;
    if (s.status < 0 && (st->status >= 0 || s.status < st->status)) st->status = s.status;
}

// SELL-32 row loop over the 2 x 2 blocks of the node pattern: f(value block, column) for the row's entries
template <class F>
__device__ __forceinline__ void block_row(const int32_t* sp, const int32_t* sc, const int16_t* sc16, int row,
                                          const F& f) {
    const int s = row >> 5, lane = row & 31;
    const int base = __ldg(sp + s), w = (__ldg(sp + s + 1) - base) >> 5;
    for (int k = 0; k < w; ++k) {
        const int pos = base + 32 * k + lane;
        const int col = sc16 ? row + (int)__ldg(sc16 + pos) : __ldg(sc + pos);
        f(pos, col);
    }
}

// r_T -= J_TV z_V (the T-V blocks: entry 2 of each 2 x 2 block)
__global__ void __launch_bounds__(kThreads) k_fg_couple(int N, const int32_t* __restrict__ sp,
                                                        const int32_t* __restrict__ sc,
                                                        const int16_t* __restrict__ sc16,
                                                        const double* __restrict__ vals4,
                                                        const double* __restrict__ zV, double* __restrict__ rT,
                                                        const FgState* st) {
    if (skipped(st)) return;
    const int row = blockIdx.x * kThreads + threadIdx.x;
    if (row >= N) return;
    double acc = 0.0;
    block_row(sp, sc, sc16, row, [&](int pos, int col) { acc = fma(__ldg(vals4 + 4 * (size_t)pos + 2), zV[col], acc); });
    rT[row] -= acc;
}

// w = J z with z = (z_V, z_T) interleaved, which is also stored as the preconditioned vector Z_j
__global__ void __launch_bounds__(kThreads) k_fg_spmv(int N, const int32_t* __restrict__ sp,
                                                      const int32_t* __restrict__ sc, const int16_t* __restrict__ sc16,
                                                      const double* __restrict__ vals4, const double* __restrict__ zV,
                                                      const double* __restrict__ zT, double* __restrict__ w,
                                                      double* __restrict__ Zj, const FgState* st) {
    if (skipped(st)) return;
    const int row = blockIdx.x * kThreads + threadIdx.x;
    if (row >= N) return;
    double aV = 0.0, aT = 0.0;
    block_row(sp, sc, sc16, row, [&](int pos, int col) {
        const double2 m01 = __ldg(reinterpret_cast<const double2*>(vals4) + 2 * (size_t)pos);
        const double2 m23 = __ldg(reinterpret_cast<const double2*>(vals4) + 2 * (size_t)pos + 1);
        const double v = zV[col], t = zT[col];
        aV = fma(m01.x, v, fma(m01.y, t, aV));
        aT = fma(m23.x, v, fma(m23.y, t, aT));
    });
    reinterpret_cast<double2*>(w)[row] = make_double2(aV, aT);
    reinterpret_cast<double2*>(Zj)[row] = make_double2(zV[row], zT[row]);
}

}  // namespace

namespace {

// Givens rotations on column j (its new subdiagonal entry hn), the residual estimate |g_{j+1}| and the stopping
// test |g_{j+1}| <= eta beta (one thread)
__device__ void finish_column(FgState* st, double* hj, int j, double hn) {
    for (int i = 0; i < j; ++i) {
        const double t = st->cs[i] * hj[i] + st->sn[i] * hj[i + 1];
        hj[i + 1] = -st->sn[i] * hj[i] + st->cs[i] * hj[i + 1];
        hj[i] = t;
    }
    const double den = hypot(hj[j], hn);
    const double c = den > 0.0 ? hj[j] / den : 1.0, s = den > 0.0 ? hn / den : 0.0;
    st->cs[j] = c;
    st->sn[j] = s;
    hj[j] = den;
    hj[j + 1] = 0.0;
    st->g[j + 1] = -s * st->g[j];
    st->g[j] = c * st->g[j];
    st->outer = j + 1;
    const bool converged = fabs(st->g[j + 1]) <= st->eta * st->beta;
    if (converged || j + 1 == kFgMax || !(hn > 0.0)) {
        st->done = 1;
        st->k = j + 1;
    } else {
        st->scale = 1.0 / hn;
    }
}

// Gram-Schmidt coefficients of outer iteration j from a dots launch over V_0..V_j (slot j + 1: (w, w)). Pass 1:
// h_ij = (w, v_i); when (w, w) - sum h_ij^2 keeps at least kReorth of (w, w) that is the new vector's squared
// norm and the column is finished (single pass). Otherwise pass 2 (after w -= sum h_ij v_i): the corrections
// c_i = (w, v_i) are added to h_ij and the norm is sqrt((w, w) - sum c_i^2). The sums in a fixed order, the rest
// on one thread.
constexpr double kReorth = 0.01;
__global__ void k_fg_gs(FgState* st, const double* partial, int G, int j, int pass) {
    if (skipped(st) || (pass == 2 && st->single)) return;
    // the j + 2 block-partial sums, one warp per quantity (lanes take every 32nd block, then a fixed shuffle tree)
    __shared__ double tot[kDots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp <= j + 1) {
        double v = 0.0;
        for (int b = lane; b < G; b += 32) v += partial[(size_t)warp * G + b];
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) tot[warp] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double* hj = st->h + (size_t)j * (kFgMax + 1);
    const double ww = tot[j + 1];
    if (!isfinite(ww)) {
        st->status = RAFEM_ERR_NONFINITE;
        st->done = 1;
        st->k = 0;
        return;
    }
    double c2 = 0.0;
    for (int i = 0; i <= j; ++i) {
        const double c = tot[i];
        st->coef[i] = c;
        hj[i] = pass == 1 ? c : hj[i] + c;
        c2 = fma(c, c, c2);
    }
    const double nh2 = ww - c2;
    if (pass == 1) {
        st->single = nh2 >= kReorth * ww;
        if (!st->single) return;
    }
    finish_column(st, hj, j, sqrt(fmax(nh2, 0.0)));
}

// w -= sum_{i <= j} coef_i V_i. The result scaled by 1 / its norm goes to next (the basis vector j + 1) after the
// column's last pass (pass 1 when it was the only one, else pass 2); after a first pass that needs a second, w is
// updated in place.
__global__ void __launch_bounds__(kThreads) k_fg_sub(int n2, double* __restrict__ w, const double* __restrict__ V,
                                                     size_t ld, int j, const FgState* st, double* __restrict__ next,
                                                     int pass) {
    if (skipped(st) || (pass == 2 && st->single)) return;
    const bool last = pass == 2 || st->single;
    double c[kFgMax + 1];
#pragma unroll
    for (int i = 0; i <= kFgMax; ++i) c[i] = i <= j ? st->coef[i] : 0.0;
    const double sc = st->scale;
    for (int k = blockIdx.x * kThreads + threadIdx.x; k < n2; k += gridDim.x * kThreads) {
        double v = w[k];
#pragma unroll
        for (int i = 0; i <= kFgMax; ++i)
            if (i <= j) v = fma(-c[i], V[i * ld + k], v);
        if (last)
            next[k] = v * sc;
        else
            w[k] = v;
    }
}

// y = R^-1 g over the k columns; the solve's statistics into the two instance states (iterations of the inner
// solves, outer iterations as refinements, the relative residual estimate |g_k| / beta)
__global__ void k_fg_solve(FgState* st, InstState* instV, InstState* instT) {
    const int k = st->k;
    for (int i = k - 1; i >= 0; --i) {
        double t = st->g[i];
        for (int l = i + 1; l < k; ++l) t -= st->h[(size_t)l * (kFgMax + 1) + i] * st->y[l];
        const double d = st->h[(size_t)i * (kFgMax + 1) + i];
        st->y[i] = d != 0.0 ? t / d : 0.0;
    }
    InstState v{}, t{};
    v.iters = st->itV;
    v.refine = st->outer;
    v.status = st->status;
    v.relres = st->beta > 0.0 ? fabs(st->g[k]) / st->beta : 0.0;
    t.iters = st->itT;
    t.status = st->status;
    t.relres = v.relres;
    instV[0] = v;
    instT[0] = t;
}

// delta = sum_{i < k} y_i Z_i (the correction of the Newton iteration)
__global__ void __launch_bounds__(kThreads) k_fg_update(int n2, const double* __restrict__ Z, size_t ld,
                                                        const FgState* st, double* __restrict__ delta) {
    const int k = st->k;
    double y[kFgMax];
#pragma unroll
    for (int i = 0; i < kFgMax; ++i) y[i] = i < k ? st->y[i] : 0.0;
    for (int q = blockIdx.x * kThreads + threadIdx.x; q < n2; q += gridDim.x * kThreads) {
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < kFgMax; ++i)
            if (i < k) v = fma(y[i], Z[i * ld + q], v);
        delta[q] = v;
    }
}

}  // namespace

// blocks of the grid-stride 2N-vector kernels and of the dots partials: two per SM
int fg_grid() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return 2 * sms;
}

cudaError_t launch_fg_dots(int n2, const double* w, const double* V, size_t ld, int nv, const FgState* st,
                           double* partial, int G, cudaStream_t s, int pass) {
    if (nv < 0 || nv > kFgMax + 1) return cudaErrorInvalidValue;
    k_fg_dots<<<G, kThreads, 0, s>>>(n2, w, V, ld, nv, st, partial, pass);
    return cudaGetLastError();
}

cudaError_t launch_fg_init(FgState* st, const double* partial, int G, double* newton_rr, double tol, cudaStream_t s) {
    k_fg_init<<<1, 32, 0, s>>>(st, partial, G, newton_rr, tol);
    return cudaGetLastError();
}

cudaError_t launch_fg_scale(int n2, const double* src, double* dst, const FgState* st, cudaStream_t s) {
    k_fg_scale<<<fg_grid(), kThreads, 0, s>>>(n2, src, dst, st);
    return cudaGetLastError();
}

cudaError_t launch_fg_split(int N, const double* v, double* rV, double* rT, double* zV, double* zT,
                            const FgState* st, cudaStream_t s) {
    k_fg_split<<<fg_grid(), kThreads, 0, s>>>(N, v, rV, rT, zV, zT, st);
    return cudaGetLastError();
}

cudaError_t launch_fg_count(FgState* st, const InstState* inst, int which, cudaStream_t s) {
    k_fg_count<<<1, 1, 0, s>>>(st, inst, which);
    return cudaGetLastError();
}

cudaError_t launch_fg_couple(int N, const int32_t* sp, const int32_t* sc, const int16_t* sc16, const double* vals4,
                             const double* zV, double* rT, const FgState* st, cudaStream_t s) {
    k_fg_couple<<<blocks_for(N), kThreads, 0, s>>>(N, sp, sc, sc16, vals4, zV, rT, st);
    return cudaGetLastError();
}

cudaError_t launch_fg_spmv(int N, const int32_t* sp, const int32_t* sc, const int16_t* sc16, const double* vals4,
                           const double* zV, const double* zT, double* w, double* Zj, const FgState* st,
                           cudaStream_t s) {
    k_fg_spmv<<<blocks_for(N), kThreads, 0, s>>>(N, sp, sc, sc16, vals4, zV, zT, w, Zj, st);
    return cudaGetLastError();
}

cudaError_t launch_fg_gs(FgState* st, const double* partial, int G, int j, int pass, cudaStream_t s) {
    if (j < 0 || j >= kFgMax) return cudaErrorInvalidValue;
    k_fg_gs<<<1, 32 * kDots, 0, s>>>(st, partial, G, j, pass);
    return cudaGetLastError();
}

cudaError_t launch_fg_sub(int n2, double* w, const double* V, size_t ld, int j, const FgState* st, double* next,
                          int pass, cudaStream_t s) {
    if (j < 0 || j >= kFgMax || !next) return cudaErrorInvalidValue;
    k_fg_sub<<<fg_grid(), kThreads, 0, s>>>(n2, w, V, ld, j, st, next, pass);
    return cudaGetLastError();
}

cudaError_t launch_fg_finish(int n2, const double* Z, size_t ld, FgState* st, double* delta, InstState* instV,
                             InstState* instT, cudaStream_t s) {
    k_fg_solve<<<1, 1, 0, s>>>(st, instV, instT);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fg_update<<<fg_grid(), kThreads, 0, s>>>(n2, Z, ld, st, delta);
    return cudaGetLastError();
}

}  // namespace rafem
