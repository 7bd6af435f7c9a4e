// ILU(0)-preconditioned conjugate gradients (Sec. II-B: CG for symmetric positive-definite systems, with a
// preconditioner to speed up convergence).
//
// The factorisation is taken on a symmetric permutation P A P^T whose rows are grouped into levels that never
// depend on each other (greedy colours of the matrix graph, or dependency levels of the original numbering;
// setup.h build_ilu). Each level is a contiguous, 32-aligned range of rows of a SELL-32 layout, so every
// triangular sweep is a sequence of level passes: all rows of a level at once (one thread per row, coalesced
// slice loads), a grid barrier between levels.
//
// Numeric ILU(0) (once per assembled matrix): the row-by-row IKJ form, one thread per row of a level, levels in
// order (one launch each). Row i reads only rows of earlier levels, which are final.
//
// Solve (one persistent cooperative launch, all iterations), in the permuted numbering:
//   phase A (all rows):   p = z + beta p,  q = A z + beta q  (= A p),  partial sums of delta = (p, q)
//   -- barrier --         alpha = gamma / delta
//   phase B (all rows):   x += alpha p,  r -= alpha q,  partial rr;  level-0 rows: z = r
//   -- barrier --         convergence test on rr
//   forward levels 1..C-1:  z_i = r_i - sum_{j<i} L_ij z_j      (the last level also divides by u_ii)
//   backward levels C-2..0: z_i = (z_i - sum_{j>i} U_ij z_j) / u_ii;  partial sums of gamma = (r, z)
//   -- a barrier after each level; after level 0: beta = gamma / gamma_prev --
// Every slice is always handled by the same warp, so row-local vectors stay with their thread; reads of other
// rows' values written during the launch go through L2. Sums are reduced in a fixed order by every block
// (deterministic), and every barrier wait is bounded.
#include <cuda_runtime.h>

#include <cmath>

#include "grid_sync.cuh"
#include "internal.h"

namespace rafem {

namespace {

constexpr int kIluBlock = 512;
constexpr int kIluWarps = kIluBlock / 32;
constexpr int kThreads = 256;

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

struct Lay {
    int Np, n_levels;
    const int32_t* lvl;
    const int32_t* sp;
    const int32_t* sc;
    const uint8_t* rlen;
    const uint8_t* dk;
    const int32_t* perm;
};

Lay lay_of(const IluLayout& L) { return Lay{L.Np, L.n_levels, L.lvl, L.sp, L.sc, L.rlen, L.dk, L.perm}; }

// ---- refactorisation ----------------------------------------------------------------------------------------

__global__ void k_ilu_init(long long nnz, const int32_t* __restrict__ pmap, const double* __restrict__ vals,
                           double* __restrict__ Ap, double* __restrict__ F) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        const int pm = pmap[q];
        const double v = pm >= 0 ? vals[pm] : (pm == -2 ? 1.0 : 0.0);
        Ap[q] = v;
        F[q] = v;
    }
}

// IKJ ILU(0) of the rows of one level (slices [s0, s1)): for each stored k < i in increasing order
// l_ik = w_k / u_kk, then w_j -= l_ik u_kj for the stored j > k of row k that row i also stores.
__global__ void __launch_bounds__(kThreads) k_ilu_factor(Lay L, double* __restrict__ F, int s0, int s1) {
    const int s = s0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31, row = s * 32 + lane;
    const int len = L.rlen[row], d = L.dk[row], base = L.sp[s];
    for (int k = 0; k < d; ++k) {
        const int pos = base + 32 * k + lane;
        const int c = L.sc[pos];
        const int cl = c & 31, cb = L.sp[c >> 5], cd = L.dk[c], clen = L.rlen[c];
        const double l = F[pos] / F[cb + 32 * cd + cl];
        F[pos] = l;
        int p = k + 1;
        int cp = p < len ? L.sc[base + 32 * p + lane] : 0x7fffffff;
        for (int t = cd + 1; t < clen && p < len; ++t) {
            const int j = L.sc[cb + 32 * t + cl];
            while (cp < j) {
                ++p;
                cp = p < len ? L.sc[base + 32 * p + lane] : 0x7fffffff;
            }
            if (cp == j) F[base + 32 * p + lane] -= l * F[cb + 32 * t + cl];
        }
    }
}

// dinv_i = 1 / u_ii for every padded row (the sweeps multiply instead of dividing: an FP64 division costs about
// ten FP64 operations on a part whose FP64 rate is a small fraction of its FP32 rate)
__global__ void k_ilu_dinv(Lay L, const double* __restrict__ F, double* __restrict__ dinv) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= L.Np) return;
    dinv[row] = 1.0 / F[L.sp[row >> 5] + 32 * L.dk[row] + (row & 31)];
}

// ---- standalone application z = (LU)^-1 r ------------------------------------------------------------------

__global__ void k_ilu_gather(int Np, const int32_t* __restrict__ perm, const double* __restrict__ r,
                             double* __restrict__ rv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Np) rv[i] = perm[i] >= 0 ? r[perm[i]] : 0.0;
}

__global__ void k_ilu_scatter(int Np, const int32_t* __restrict__ perm, const double* __restrict__ zv,
                              double* __restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Np && perm[i] >= 0) z[perm[i]] = zv[i];
}

// forward pass of one level: z = rv - L z (lower entries); `last` also divides by the diagonal
__global__ void k_ilu_fwd(Lay L, const double* __restrict__ F, const double* __restrict__ dinv,
                          const double* __restrict__ rv, double* __restrict__ z, int s0, int s1, int last) {
    const int s = s0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31, row = s * 32 + lane, base = L.sp[s], d = L.dk[row];
    double acc = rv[row];
    for (int k = 0; k < d; ++k) {
        const int pos = base + 32 * k + lane;
        acc -= F[pos] * z[L.sc[pos]];
    }
    if (last) acc *= dinv[row];
    z[row] = acc;
}

// backward pass of one level (not the last): z = (z - U z) / u_ii (upper entries)
__global__ void k_ilu_bwd(Lay L, const double* __restrict__ F, const double* __restrict__ dinv, double* __restrict__ z,
                          int s0, int s1) {
    const int s = s0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (s >= s1) return;
    const int lane = threadIdx.x & 31, row = s * 32 + lane, base = L.sp[s], d = L.dk[row], len = L.rlen[row];
    double acc = z[row];
    for (int k = d + 1; k < len; ++k) {
        const int pos = base + 32 * k + lane;
        acc -= F[pos] * z[L.sc[pos]];
    }
    z[row] = acc * dinv[row];
}

// ---- persistent PCG ----------------------------------------------------------------------------------------

struct Args {
    Lay L;
    const double* A;
    const double* F;
    const double* dinv;
    const double* b;
    double* x;
    double *xv, *bv, *r, *z, *p, *q;
    double* partial;
    GridBarrier* bar;
    InstState* inst;
    double tol;
    int max_iter;
    long long spin_limit_ns;
};

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ double* slot(const Args& a, int k) { return a.partial + (size_t)k * gridDim.x; }

// Slices [s0, s1) handled by this warp: slice s always belongs to warp (s mod total warps), in every phase.
template <class Fn>
__device__ __forceinline__ void for_slices(int s0, int s1, const Fn& f) {
    const int tw = gridDim.x * kIluWarps;
    const int gw = blockIdx.x * kIluWarps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    int s = s0 + ((gw - s0 % tw) % tw + tw) % tw;
    for (; s < s1; s += tw) f(s, s * 32 + lane, lane);
}

// Block sums of NQ values (fixed order) written to part[q][blockIdx.x]. Consecutive phases use disjoint slot
// ranges of the partial buffer (slots 0 | 1-2 | 3 | 4), so a fast block publishing the next phase's sums never
// overwrites sums a slower block is still reading.
template <int NQ>
__device__ __forceinline__ void publish(const double (&v)[NQ], double* sm, double* part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) sm[q * kIluBlock + threadIdx.x] = v[q];
    __syncthreads();
    if (warp < NQ) {
        double acc = sm[warp * kIluBlock + lane];
#pragma unroll
        for (int k = 1; k < kIluWarps; ++k) acc += sm[warp * kIluBlock + 32 * k + lane];
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[(size_t)warp * gridDim.x + blockIdx.x] = acc;
    }
}

// After a barrier: every block sums the per-block partials of NQ quantities in the same order.
template <int NQ>
__device__ __forceinline__ void totals(const double* partial, double* s_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < NQ) {
        double acc = 0.0;
        for (int t = lane; t < (int)gridDim.x; t += 32) acc += ldcg(partial + (size_t)warp * gridDim.x + t);
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_tot[warp] = acc;
    }
    __syncthreads();
}

// sum over stored entries k in [k0, k1) of M[pos] * v[col], in order. Values and columns are loaded in batches of
// kBatch before the gathers that depend on them, so a row waits for two memory round trips per batch instead of
// two per entry (a level pass is latency-bound otherwise).
constexpr int kBatch = 8;
__device__ __forceinline__ double row_dot(const Lay& L, const double* __restrict__ M, const double* v, int base,
                                          int lane, int k0, int k1) {
    double acc = 0.0;
    for (int k = k0; k < k1; k += kBatch) {
        double m[kBatch], x[kBatch];
        int c[kBatch];
#pragma unroll
        for (int t = 0; t < kBatch; ++t) {
            const int pos = base + 32 * (k + t) + lane;
            const bool ok = k + t < k1;
            m[t] = ok ? __ldg(M + pos) : 0.0;
            c[t] = ok ? __ldg(L.sc + pos) : -1;
        }
#pragma unroll
        for (int t = 0; t < kBatch; ++t) x[t] = c[t] >= 0 ? ldcg(v + c[t]) : 0.0;
#pragma unroll
        for (int t = 0; t < kBatch; ++t) acc = fma(m[t], x[t], acc);
    }
    return acc;
}

__global__ void __launch_bounds__(kIluBlock, 1) k_ilu_pcg(Args a) {
    __shared__ double sm[3 * kIluBlock];
    __shared__ double s_tot[4];
    const Lay& L = a.L;
    const int S = L.Np / 32, C = L.n_levels;
    const int s_l0 = L.lvl[1] / 32;
    unsigned target = 0;
    bool err = false;
    double bb = 0.0, rr = 0.0, gamma = 0.0, beta = 0.0, alpha = 0.0;
    int iters = 0, status = RAFEM_NOT_CONVERGED;

    // gather x, b into the level order; ||b||^2
    {
        double v[1] = {0.0};
        for_slices(0, S, [&](int, int row, int) {
            const int o = L.perm[row];
            const double bi = o >= 0 ? a.b[o] : 0.0;
            a.xv[row] = o >= 0 ? a.x[o] : 0.0;
            a.bv[row] = bi;
            v[0] = fma(bi, bi, v[0]);
        });
        publish<1>(v, sm, slot(a, 0));
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        totals<1>(slot(a, 0), s_tot);
        bb = s_tot[0];
    }
    const double thr = a.tol * a.tol * (bb > 0.0 ? bb : 1.0);
    // r = b - A x; level-0 rows start the forward pass
    if (!err) {
        double v[2] = {0.0, 0.0};
        for_slices(0, S, [&](int s, int row, int lane) {
            const int base = __ldg(L.sp + s);
            const double ri = a.bv[row] - row_dot(L, a.A, a.xv, base, lane, 0, __ldg(L.rlen + row));
            a.r[row] = ri;
            v[0] = fma(ri, ri, v[0]);
            if (s < s_l0) {
                double zi = ri;
                if (C == 1) {
                    zi = ri * __ldg(a.dinv + row);
                    v[1] = fma(ri, zi, v[1]);
                }
                a.z[row] = zi;
            }
        });
        publish<2>(v, sm, slot(a, 1));
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        totals<2>(slot(a, 1), s_tot);
        rr = s_tot[0];
        gamma = s_tot[1];
    }
    bool done = err || !(rr > thr);
    if (!err && !(rr == rr)) status = RAFEM_ERR_NONFINITE;
    else if (done) status = RAFEM_OK;
    // z = (LU)^-1 r for the levels after the first; gamma = (r, z)
    auto precondition = [&]() -> bool {
        double g[1] = {0.0};
        for (int l = 1; l < C; ++l) {
            const bool last = l == C - 1;
            for_slices(L.lvl[l] / 32, L.lvl[l + 1] / 32, [&](int s, int row, int lane) {
                const int base = __ldg(L.sp + s), d = __ldg(L.dk + row);
                const double ri = ldcg(a.r + row);
                double zi = ri - row_dot(L, a.F, a.z, base, lane, 0, d);
                if (last) {
                    zi *= __ldg(a.dinv + row);
                    g[0] = fma(ri, zi, g[0]);
                }
                a.z[row] = zi;
            });
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) return false;
        }
        for (int l = C - 2; l >= 0; --l) {
            for_slices(L.lvl[l] / 32, L.lvl[l + 1] / 32, [&](int s, int row, int lane) {
                const int base = __ldg(L.sp + s), d = __ldg(L.dk + row), len = __ldg(L.rlen + row);
                const double zi =
                    (ldcg(a.z + row) - row_dot(L, a.F, a.z, base, lane, d + 1, len)) * __ldg(a.dinv + row);
                a.z[row] = zi;
                g[0] = fma(ldcg(a.r + row), zi, g[0]);
            });
            if (l == 0) publish<1>(g, sm, slot(a, 3));
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) return false;
        }
        totals<1>(slot(a, 3), s_tot);
        return true;
    };
    if (!done && C > 1) {
        if (!precondition()) err = true;
        else gamma = s_tot[0];
    }
    bool first = true;
    while (!done && !err) {
        if (!(gamma > 0.0)) {
            status = gamma == gamma ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
            break;
        }
        // phase A: p = z + beta p, q = A z + beta q, delta = (p, q)
        {
            double v[1] = {0.0};
            const double bt = first ? 0.0 : beta;
            for_slices(0, S, [&](int s, int row, int lane) {
                const int base = __ldg(L.sp + s);
                const double az = row_dot(L, a.A, a.z, base, lane, 0, __ldg(L.rlen + row));
                const double zi = ldcg(a.z + row);
                const double pi = first ? zi : fma(bt, a.p[row], zi);
                const double qi = first ? az : fma(bt, a.q[row], az);
                a.p[row] = pi;
                a.q[row] = qi;
                v[0] = fma(pi, qi, v[0]);
            });
            publish<1>(v, sm, slot(a, 0));
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<1>(slot(a, 0), s_tot);
            const double delta = s_tot[0];
            if (!(delta > 0.0)) {
                status = delta == delta ? RAFEM_ERR_BREAKDOWN : RAFEM_ERR_NONFINITE;
                break;
            }
            alpha = gamma / delta;
            first = false;
        }
        // phase B: x += alpha p, r -= alpha q, rr; level-0 rows: z = r
        {
            double v[2] = {0.0, 0.0};
            for_slices(0, S, [&](int s, int row, int lane) {
                a.xv[row] = fma(alpha, a.p[row], a.xv[row]);
                const double ri = fma(-alpha, a.q[row], a.r[row]);
                a.r[row] = ri;
                v[0] = fma(ri, ri, v[0]);
                if (s < s_l0) {
                    double zi = ri;
                    if (C == 1) {
                        zi = ri * __ldg(a.dinv + row);
                        v[1] = fma(ri, zi, v[1]);
                    }
                    a.z[row] = zi;
                }
            });
            publish<2>(v, sm, slot(a, 1));
            if (grid_barrier(a.bar, a.spin_limit_ns, target)) { err = true; break; }
            totals<2>(slot(a, 1), s_tot);
            rr = s_tot[0];
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
        const double gprev = gamma;
        if (C > 1) {
            if (!precondition()) { err = true; break; }
        }
        gamma = s_tot[C > 1 ? 0 : 1];
        beta = gamma / gprev;
    }
    // true residual and the solution back in the original ordering
    double relres = 0.0;
    if (!err) {
        double v[1] = {0.0};
        for_slices(0, S, [&](int s, int row, int lane) {
            const int base = __ldg(L.sp + s);
            const double ri = a.bv[row] - row_dot(L, a.A, a.xv, base, lane, 0, __ldg(L.rlen + row));
            v[0] = fma(ri, ri, v[0]);
            const int o = L.perm[row];
            if (o >= 0) a.x[o] = ldcg(a.xv + row);
        });
        publish<1>(v, sm, slot(a, 4));
        err = grid_barrier(a.bar, a.spin_limit_ns, target);
        totals<1>(slot(a, 4), s_tot);
        relres = sqrt(s_tot[0] / (bb > 0.0 ? bb : 1.0));
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

}  // namespace

cudaError_t launch_ilu_refactor(const IluLayout& L, const double* vals, double* Ap, double* F, double* dinv,
                                cudaStream_t st) {
    k_ilu_init<<<148 * 8, kThreads, 0, st>>>(L.nnz, L.pmap, vals, Ap, F);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const Lay lay = lay_of(L);
    for (int l = 1; l < L.n_levels; ++l) {
        const int s0 = L.h_lvl[l] / 32, s1 = L.h_lvl[l + 1] / 32;
        if (s1 <= s0) continue;
        k_ilu_factor<<<blocks_for(32LL * (s1 - s0)), kThreads, 0, st>>>(lay, F, s0, s1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_ilu_dinv<<<blocks_for(L.Np), kThreads, 0, st>>>(lay, F, dinv);
    return cudaGetLastError();
}

int ilu_max_blocks(int* block_threads) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ilu_pcg, kIluBlock, 0) != cudaSuccess) return 0;
    *block_threads = kIluBlock;
    return sms * (per < 2 ? per : 2);
}

cudaError_t launch_ilu_pcg(const IluSolveArgs& s, int grid, cudaStream_t st) {
    Args a{lay_of(*s.L), s.A, s.F, s.dinv, s.b, s.x, s.xv, s.bv, s.r, s.z, s.p, s.q, s.partial, s.bar, s.inst,
           s.tol, s.max_iter, s.spin_limit_ns};
    cudaError_t e = cudaMemsetAsync(s.bar, 0, sizeof(GridBarrier), st);
    if (e != cudaSuccess) return e;
    if (s.bar_missing > 0 && (e = launch_barrier_reset(s.bar, s.bar_missing, st)) != cudaSuccess) return e;
    void* params[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)k_ilu_pcg, dim3(grid), dim3(kIluBlock), params, 0, st);
}

cudaError_t launch_ilu_apply(const IluLayout& L, const double* F, const double* dinv, const double* r, double* z,
                             double* rv, double* zv, cudaStream_t st) {
    const Lay lay = lay_of(L);
    k_ilu_gather<<<blocks_for(L.Np), kThreads, 0, st>>>(L.Np, L.perm, r, rv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int C = L.n_levels;
    for (int l = 0; l < C; ++l) {
        const int s0 = L.h_lvl[l] / 32, s1 = L.h_lvl[l + 1] / 32;
        if (s1 > s0) k_ilu_fwd<<<blocks_for(32LL * (s1 - s0)), kThreads, 0, st>>>(lay, F, dinv, rv, zv, s0, s1,
                                                                           l == C - 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int l = C - 2; l >= 0; --l) {
        const int s0 = L.h_lvl[l] / 32, s1 = L.h_lvl[l + 1] / 32;
        if (s1 > s0) k_ilu_bwd<<<blocks_for(32LL * (s1 - s0)), kThreads, 0, st>>>(lay, F, dinv, zv, s0, s1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_ilu_scatter<<<blocks_for(L.Np), kThreads, 0, st>>>(L.Np, L.perm, zv, z);
    return cudaGetLastError();
}

}  // namespace rafem
